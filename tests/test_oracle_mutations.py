"""Mutation check of the oracle pins: each plausible slip, planted in a copy of
``oracle.c`` compiled on the CPU, must make at least one pin of
``test_oracle_pins.py`` fail.  The real oracle is never modified."""
import inspect
import os

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.lib_path()), "oracle.c")

MUTANTS = [
    # Sect. 2.3 pair force, jerk, potential
    ("jerk coefficient 3 -> 2", "- 3.0 * rv * rx / s5", "- 2.0 * rv * rx / s5"),
    ("jerk sign of radial term", "jy += m * (uy / s3 - 3.0", "jy += m * (uy / s3 + 3.0"),
    ("acc power s^3 -> s^2", "ax += m * rx / s3;", "ax += m * rx / s2;"),
    ("separation operands swapped", "double rz = xj[3 * j + 2] - xi[3 * i + 2];\n            double ux",
     "double rz = xi[3 * i + 2] - xj[3 * j + 2];\n            double ux"),
    ("velocity difference swapped", "double uz = vj[3 * j + 2] - vi[3 * i + 2];",
     "double uz = vi[3 * i + 2] - vj[3 * j + 2];"),
    ("softening dropped", "double s2 = r2 + eps2;", "double s2 = r2;"),
    ("potential sign", "phi -= m / s;", "phi += m / s;"),
    ("potential power", "phi -= m / s;", "phi -= m / s2;"),
    ("self skipped by position", "if (idx_j[j] == idx_i[i])\n                continue;                               /* self-interaction */",
     "if (j == i)\n                continue;"),
    ("mass dropped from jerk", "jx += m * (ux / s3", "jx += (ux / s3"),
    # Sect. 2.5 nearest neighbour
    ("nn tie to later j", "if (r2 < best) {", "if (r2 <= best) {"),
    ("nn on softened distance", "if (r2 < best) {\n                best = r2;", "if (s2 < best) {\n                best = s2;"),
    # Sect. 4 neighbour lists
    ("list radius not strict", "if (r2 < h2[i]) {", "if (r2 <= h2[i]) {"),
    ("list overflow not counted", "if (cnt > maxnb)\n            ++overflowed;", "if (cnt > maxnb + 1)\n            ++overflowed;"),
    # Sect. 2.2 predictor, Eq. 1 and Eq. 2
    ("Eq. 1 jerk term /6 -> /2", "j * dt * dt * dt / 6.0", "j * dt * dt * dt / 2.0"),
    ("Eq. 1 acc term halving dropped", "a * dt * dt / 2.0 + j", "a * dt * dt + j"),
    ("Eq. 2 jerk term /2 -> /6", "vp[3 * k + c] = v + a * dt + j * dt * dt / 2.0;",
     "vp[3 * k + c] = v + a * dt + j * dt * dt / 6.0;"),
    ("predictor ignores tj", "double dt = t - tj[k];", "double dt = t;"),
    # Hermite corrector and time steps
    ("corrector a0-a1 sign", "double d2 = (-6.0 * (a0[c] - a1[c])", "double d2 = (-6.0 * (a1[c] - a0[c])"),
    ("corrector jerk weights swapped", "dt * (4.0 * j0[c] + 2.0 * j1[c])", "dt * (2.0 * j0[c] + 4.0 * j1[c])"),
    ("corrector dt^5/120 -> /24", "d3 * dt5 / 120.0", "d3 * dt5 / 24.0"),
    ("corrector v term /6 -> /2", "d2 * dt3 / 6.0", "d2 * dt3 / 2.0"),
    ("aarseth |j|^2 -> |j|", "(na * n2 + nj * nj)", "(na * n2 + nj)"),
    ("aarseth a2 -> a3", "(na * n2 + nj * nj)", "(na * n3 + nj * nj)"),
    ("block dt doubles past dt_max", "&& 2.0 * dt <= dt_max", ""),
    ("block dt commensurability", "fmod(t, 2.0 * dt) == 0.0", "fmod(t, dt) == 0.0"),
    ("integrator i not predicted", "memcpy(&xa[3 * q], &xp[3 * k], 3 * sizeof(double));",
     "memcpy(&xa[3 * q], &x[3 * k], 3 * sizeof(double));"),
    ("corrector applied to old position", "orc_hermite_correct(h, &xp[3 * k], &vp[3 * k]",
     "orc_hermite_correct(h, &x[3 * k], &vp[3 * k]"),
    # Sect. 3.2 energy
    ("kinetic energy factor", "kin += 0.5 * m[i]", "kin += m[i]"),
    ("energy pair loop includes j == i", "for (long j = i + 1; j < n; ++j) {\n            double rx = x[3 * j] - x[3 * i];",
     "for (long j = i; j < n; ++j) {\n            double rx = x[3 * j] - x[3 * i];"),
]


def _pin_calls():
    calls = []
    for name, fn in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        params = list(inspect.signature(fn).parameters)
        if params[:1] != ["orc"]:
            continue
        if name == "test_two_body_closed_form":
            calls += [(name + "[0]", lambda o, f=fn: f(o, 0.0)),
                      (name + "[eps]", lambda o, f=fn: f(o, 0.04))]
        else:
            calls.append((name, lambda o, f=fn: f(o)))
    return calls


@pytest.mark.parametrize("label,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_every_mutant_fails_a_pin(tmp_path, label, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation site not found: " + label
    mutated = src.replace(old, new)
    path = tmp_path / "oracle_mut.c"
    path.write_text(mutated)
    lib = oracle.compile_source(str(path), str(tmp_path / "liboracle_mut.so"))
    mut = oracle.Oracle(lib)
    failed = []
    for name, call in _pin_calls():
        try:
            call(mut)
        except Exception:       # assertion or numerical blow-up
            failed.append(name)
    assert failed, "no pin catches mutant: " + label
