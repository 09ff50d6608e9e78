"""Planted mistakes in a copy of the oracle must each fail at least one pin.

Each case copies the oracle source to a temporary directory, applies one
textual change (a dropped term, a flipped sign, a wrong index, a swapped
operand), compiles it and runs the pin suite against it.  This shows the pins
are strong enough to catch plausible errors in every part of the oracle.
"""
import os
import shutil

import pytest

import pins
from oracle import oracle as OR

MUTANTS = [
    ("Q+ numerator sign", "double qp = (0.5 - e0)", "double qp = (0.5 + e0)"),
    ("Q+ denominator neighbour", "(1.0 + (ep - e0))", "(1.0 + (em - e0))"),
    ("Q- denominator sign", "(1.0 - (em - e0))", "(1.0 + (em - e0))"),
    ("transport diffusion sign", "double v = (t1 - t2)", "double v = (t2 - t1)"),
    ("transport weight", "(qp + qm) * U[j]", "(qp * qm) * U[j]"),
    ("dropped source", "if (F) v = v + (0.5 * tau) * (F[j - 1] - F[j + 1]);", "if (F) v = v;"),
    ("source sign", "(F[j - 1] - F[j + 1])", "(F[j + 1] - F[j - 1])"),
    ("inner antidiffusion sign", "(dh - 0.125 *", "(dh + 0.125 *"),
    ("inner term on transported values", "((dp + dm) - 2.0 * d)", "((dhp + dhm) - 2.0 * dh)"),
    ("limiter neighbour", "fmin(fmin(sg * dhp, fabs(aph)), sg * dhm)",
     "fmin(fmin(sg * dh, fabs(aph)), sg * dhm)"),
    ("limiter dropped", "A[j] = sg * fmax(0.0, m);", "A[j] = aph;"),
    ("update sign", "UH[j] - (A[j] - A[j - 1])", "UH[j] + (A[j] - A[j - 1])"),
    ("eta ignored", "double aph = eta * (", "double aph = 0.125 * ("),
    ("half step with full lambda", "0.5 * P->lambda, P->eta", "P->lambda, P->eta"),
    ("full step transports half state", "or_line(n, old[k], w, f, P->lambda,",
     "or_line(n, half[k], w, f, P->lambda,"),
    ("half-step ghosts not refilled", "  fill_ghosts(P, axis, t, n, half, frozen);\n", "\n"),
    ("energy source without velocity", "fe[i] = p[i] * w[i];", "fe[i] = p[i];"),
    ("velocity from M/E", "v[a] = m / h;", "v[a] = m / E;"),
    ("EoS root", "sqrt(4.0 * E * E - 3.0 * M * M)", "sqrt(4.0 * E * E - 2.0 * M * M)"),
    ("baryon boost", "sqrt((ee + pp) / h)", "sqrt(ee / h)"),
    ("bag branch constant", "- 4.0 * B * E)", "- 3.0 * B * E)"),
    ("mirror parity dropped", "double par = (m < n || k != 1 + axis) ? 1.0 : -1.0;",
     "double par = 1.0;"),
    ("periodic wrap off by one", "int src = ((g % n) + n) % n;", "int src = ((g % n) + n + 1) % n;"),
    ("axis table", "{0, 1, 2, 0, 2, 1, 2, 0, 1,", "{0, 1, 2, 0, 1, 2, 2, 0, 1,"),
    ("energy definition", "E[i] = w - p;", "E[i] = w + p;"),
    ("frozen ghost side", "long edge = b + (side == 0 ? 0 : (long)(n - 1) * st);",
     "long edge = b + (side == 1 ? 0 : (long)(n - 1) * st);"),
    ("table interpolation weight", "f * (P->table[k + 1] - P->table[k])",
     "f * (P->table[k + 1] + P->table[k])"),
    ("table interval index", "if (k > P->table_n - 2) k = P->table_n - 2;",
     "if (k > P->table_n - 3) k = P->table_n - 3;"),
    ("fixed point sign", "M / (E + table_p(P, E - M * v))", "M / (E + table_p(P, E + M * v))"),
    ("fixed point stops early", "if (fabs(d) <= OR_FP_TOL) break;", "if (fabs(d) <= 1e-3) break;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    src = open(OR.SRC).read()
    assert src.count(old) >= 1, f"mutation site not found: {old!r}"
    mutated = src.replace(old, new, 1)
    cdir = tmp_path / "m"
    cdir.mkdir()
    shutil.copy(os.path.join(OR.HERE, "shasta_oracle.h"), cdir / "shasta_oracle.h")
    (cdir / "shasta_oracle.c").write_text(mutated)
    lib = OR.build(force=True, src=str(cdir / "shasta_oracle.c"), out=str(cdir / "libm.so"))
    M = OR.Oracle(lib)
    failed = []
    for pin in pins.FAST_PINS + [lambda O: pins.pin_recover_roundtrip(O, eos=OR.EOS_BAG)]:
        try:
            pin(M)
        except (AssertionError, ValueError, FloatingPointError):
            failed.append(getattr(pin, "__name__", "bag roundtrip"))
    assert failed, f"no pin caught the planted mistake '{name}'"
