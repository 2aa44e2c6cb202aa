"""The oracle's pins catch plausible mistakes: each case compiles a copy of
the oracle's C source with one planted error (a flipped sign, a dropped term,
a wrong index or operand, a pattern off by one entry), swaps it in for the
oracle, and requires at least one of the pins to fail -- an assertion of a
pin, or the oracle's own cross-check of its count and fill passes, which
raises.  The oracle itself is never changed; the copies live in a temporary
directory."""
import ctypes
import os
import shutil
import subprocess

import pytest

import oracle
import test_oracle as pins

MUTATIONS = {
    "sign of the accumulation": ("spa_values[i] += tmp_val;", "spa_values[i] -= tmp_val;"),
    "first product of every A column dropped": (
        "spa_values[i] += tmp_val;", "if (q != Acp[k]) spa_values[i] += tmp_val;"),
    "B value of the column's first entry for every entry": (
        "double tmp_val = Aval[q] * b;", "double tmp_val = Aval[q] * Bval[Bcp[j]];"),
    "row index of the product off by its A column": (
        "                    int32_t i = Arow[q];\n                    double tmp_val",
        "                    int32_t i = Arow[Acp[k]];\n                    double tmp_val"),
    "count pass skips the last entry of each B column": (
        "            for (int64_t p = Bcp[j]; p < Bcp[j + 1]; ++p) {\n                int32_t k = Brow[p];\n                for",
        "            for (int64_t p = Bcp[j]; p + 1 < Bcp[j + 1]; ++p) {\n                int32_t k = Brow[p];\n                for"),
    "backward dB from the wrong row of dC": ("s += Aval[q] * d[i];", "s += Aval[q] * d[Arow[Acp[k]]];"),
    "backward dA with A's value in place of B's": (
        "if (dAval) dAval[q] += d[i] * Bval[p];", "if (dAval) dAval[q] += d[i] * Aval[q];"),
}


def _pins():
    """The CPU pins the mutants are run against (each returns on success)."""
    yield pins.test_fig1_worked_example
    for seed in range(6):
        yield lambda seed=seed: pins.test_bruteforce_dense(seed)
    yield pins.test_identity_products_bit_exact
    yield lambda: pins.test_squared_laplacian_13_point(3)
    for seed in range(4):
        yield lambda seed=seed: pins.test_backward_bruteforce_dense(seed)
    yield pins.test_backward_adjoint_identity


def _build_mutant(tmp_path, old, new):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-o", str(lib),
                           str(path)])
    return oracle._declare(ctypes.CDLL(str(lib)))


def test_unmutated_oracle_passes_the_pins():
    for pin in _pins():
        pin()


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path, monkeypatch):
    old, new = MUTATIONS[name]
    monkeypatch.setattr(oracle, "_lib", _build_mutant(tmp_path, old, new))
    failed = []
    for pin in _pins():
        try:
            pin()
        except (AssertionError, RuntimeError):
            failed.append(pin)
    assert failed, f"no pin caught: {name}"
