"""Mutant builds of the oracle for the pin-sensitivity tests.

TEST INFRASTRUCTURE ONLY.  A pin is only worth something if a plausible
mistake in the code it pins makes it fail.  Each entry below is one such
mistake, written as text edits of ``sisph_oracle.c``: the original fragment
(which must occur exactly once in the source) and what replaces it.
``build(k)`` writes the edited source to ``_build/oracle_mutants/`` and
compiles it with the oracle's own flags into a library of its own, so the
oracle's source and ``liboracle.so`` keep a single arithmetic path.  The
tests load a mutant through ``oracle.plant_mistake(k)``.
"""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sisph_oracle.c")
_OUT = os.path.join(os.path.dirname(_HERE), "_build", "oracle_mutants")

# k: (what the mistake is, [(original fragment, replacement), ...])
MUTANTS = {
    1: ("quintic: the 15 (1-q)^5 term dropped (W and dW/dr)",
        [("if (q < 1.0) w += 15.0 * p5(1.0 - q);", "(void)q;"),
         ("if (q < 1.0) dw -= 75.0 * p4(1.0 - q);", "(void)q;")]),
    2: ("PPE source: sign of RHS flipped",
        [("rhs += -mj / (rj * P->dt) * or_dot(uij, g);",
          "rhs += mj / (rj * P->dt) * or_dot(uij, g);")]),
    3: ("wall pressure: r_wf taken as r_f - r_w",
        [("acc[k] += s->rho[j] * dx[k] * wv;", "acc[k] -= s->rho[j] * dx[k] * wv;")]),
    4: ("viscous force: factor 4 nu read as 2 nu",
        [("double visc = mj * 4.0 * P->nu / (ri + rj) * rdw / (r2 + eh2);",
          "double visc = mj * 2.0 * P->nu / (ri + rj) * rdw / (r2 + eh2);")]),
    6: ("asymm pressure gradient: p_j - p_i read as p_i - p_j",
        [("else c = -mj / (ri * rj) * (pj - pi);", "else c = -mj / (ri * rj) * (pi - pj);")]),
    7: ("artificial viscosity also between receding pairs",
        [("if (vr < 0.0) {", "if (1) {")]),
    8: ("artificial viscosity: sign flipped",
        [("fi[k] -= mj * pi_ij * g[k];", "fi[k] += mj * pi_ij * g[k];")]),
    9: ("smoothed wall normal: no zero threshold",
        [("if (mag > 1e-6)", "if (mag > 0.0)")]),
    10: ("raw wall normal: no 1/(4h) threshold",
         [("const int keep = mag >= 1.0 / (4.0 * h);", "const int keep = mag > 0.0;")]),
    11: ("artificial stress: the tensor u (x) (u~ - u) transposed",
         [("double ai = or_dot(dti, g) / ri, aj = or_dot(dtj, g) / rj;\n"
           "        for (int k = 0; k < 3; ++k) fi[k] += mj * (ui[k] * ai + uj[k] * aj);",
           "double ai = or_dot(ui, g) / ri, aj = or_dot(uj, g) / rj;\n"
           "        for (int k = 0; k < 3; ++k) fi[k] += mj * (dti[k] * ai + dtj[k] * aj);")]),
    12: ("artificial stress: the neighbour's A_j dropped",
         [("aj = or_dot(dtj, g) / rj;", "aj = 0.0 * rj;")]),
    13: ("summation density: wall neighbours left out",
         [("acc += s->m[j] * or_kernel_w(sqrt(r2), s->prm.h, s->prm.dim);",
           "if (s->kind[j] == FLUID) acc += s->m[j] * or_kernel_w(sqrt(r2), s->prm.h, s->prm.dim);")]),
    14: ("free surface: surface rows solved like interior rows",
         [("int fs = P->free_surface && (ri / P->rho0 < P->fs_ratio);", "int fs = 0;")]),
    15: ("internal-flow p_ref taken again at every step",
         [("if (!s->pref_set) {", "if (1) {")]),
    16: ("Eq. convergence: Lambda without the absolute value",
         [("double a = fabs(rhs / dg);", "double a = rhs / dg;")]),
    17: ("Eq. convergence: wall pressures counted in the sums",
         [("      if (s->kind[i] != FLUID) continue;\n"
           "      num += fabs(s->pnew[i] - s->p[i]);",
           "      num += fabs(s->pnew[i] - s->p[i]);")]),
    18: ("Eq. convergence: the algorithm listing's max(1, .) kept in the denominator",
         [("    double dd = (lam > den) ? lam : den;\n    res = (dd > 0.0) ? num / dd : num;",
           "    double dd = (lam > den) ? lam : den;\n    if (dd < 1.0) dd = 1.0;\n"
           "    res = (dd > 0.0) ? num / dd : num;")]),
    19: ("Eq. convergence: Lambda over every fluid row, free-surface rows included",
         [("      if (!s->active[i]) s->p[i] = 0.0;\n"
           "      else {\n"
           "        double a = fabs(rhs / dg);\n"
           "        if (a > lam) lam = a;\n"
           "      }",
           "      if (!s->active[i]) s->p[i] = 0.0;\n"
           "      if (dg != 0.0) {\n"
           "        double a = fabs(rhs / dg);\n"
           "        if (a > lam) lam = a;\n"
           "      }")]),
    20: ("stop test: min_iter ignored (the loop may stop after one sweep)",
         [("    if (!isfinite(res)) { bad = 1; break; }\n"
           "    if (k >= P->min_iter && res < P->tol) { conv = 1; break; }\n"
           "    if (k >= P->max_iter) break;\n  }\n  or_wall_pressure(s);",
           "    if (!isfinite(res)) { bad = 1; break; }\n"
           "    if (res < P->tol) { conv = 1; break; }\n"
           "    if (k >= P->max_iter) break;\n  }\n  or_wall_pressure(s);")]),
    21: ("external background pressure: max in place of min",
         [("fmin(10.0 * fabs(s->p[i]), s->p_ref)", "fmax(10.0 * fabs(s->p[i]), s->p_ref)")]),
    22: ("external background pressure: |p_i| read as p_i",
         [("fmin(10.0 * fabs(s->p[i]), s->p_ref)", "fmin(10.0 * s->p[i], s->p_ref)")]),
}


def source(k: int) -> str:
    """The oracle's source with mistake k planted."""
    text = open(_SRC).read()
    for old, new in MUTANTS[k][1]:
        n = text.count(old)
        if n != 1:
            raise ValueError(f"mutant {k}: fragment found {n} times: {old!r}")
        text = text.replace(old, new)
    return text


def build(k: int) -> str:
    """Compile mutant k (once per change of the oracle's source) and return
    the path of its library."""
    os.makedirs(_OUT, exist_ok=True)
    lib = os.path.join(_OUT, f"liboracle_m{k}.so")
    deps = [_SRC, os.path.join(_HERE, "sisph_oracle.h"), os.path.abspath(__file__)]
    if os.path.exists(lib) and os.path.getmtime(lib) >= max(os.path.getmtime(d) for d in deps):
        return lib
    csrc = os.path.join(_OUT, f"sisph_oracle_m{k}.c")
    with open(csrc, "w") as f:
        f.write(source(k))
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                           "-fno-fast-math", "-fPIC", "-shared", "-I", _HERE, "-o", tmp, csrc,
                           "-lm"])
    os.replace(tmp, lib)
    return lib
