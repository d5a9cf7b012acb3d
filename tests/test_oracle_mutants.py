"""The planted mistakes of the pin-sensitivity tests live in separate mutant
builds of the oracle (oracle/mutants.py); the oracle's own source and library
keep one arithmetic path."""
import ctypes
import os

import pytest

import oracle
from oracle import mutants

SRC = os.path.join(os.path.dirname(oracle.__file__), "sisph_oracle.c")


def test_oracle_source_has_no_mistake_switch():
    text = open(SRC).read()
    for word in ("plant", "mutant", "MUTANT", "mistake"):
        assert word not in text


def test_oracle_library_exports_no_mistake_hook(oracle_lib):
    lib = ctypes.CDLL(oracle.build())
    assert not hasattr(lib, "or_plant_mistake")


@pytest.mark.parametrize("k", sorted(mutants.MUTANTS))
def test_each_mutant_edits_the_source_once(k):
    text = open(SRC).read()
    edited = mutants.source(k)
    assert edited != text
    for old, _ in mutants.MUTANTS[k][1]:
        assert text.count(old) == 1


def test_planting_switches_library_and_back(oracle_lib):
    base = oracle.lib()
    oracle.plant_mistake(1)
    try:
        assert oracle.lib() is not base
        # mistake 1 drops the 15 (1-q)^5 term: W(0.5h) changes
        bad = oracle.kernel_w(0.5, 1.0, 2)
    finally:
        oracle.plant_mistake(0)
    assert oracle.lib() is base
    assert oracle.kernel_w(0.5, 1.0, 2) != bad
    with pytest.raises(KeyError):
        oracle.plant_mistake(999)
