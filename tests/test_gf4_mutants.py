"""The GF(4) oracle's pins catch planted mistakes: each case plants one mistake in a copy of
oracle/gf4.c, builds it with the oracle's flags, and requires tests/test_gf4_oracle.py to fail
against it; the unmodified copy must pass."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_gf4_oracle.py"]

MUTANTS = {
    # Eq. 2 read per Pauli: a CN message counted toward every Pauli, commuting or not
    "vn-every-pauli": ("if (f != e && anticommute(paulis[w], pauli[f])) acc += r[f];", "if (f != e) acc += r[f];"),
    # Eq. 2: the VN->CN message not extrinsic (includes the receiving check)
    "vn-not-extrinsic": ("if (f != e && anticommute(paulis[w], pauli[f])) acc += r[f];",
                         "if (anticommute(paulis[w], pauli[f])) acc += r[f];"),
    # the scalar message: commuting and anticommuting Paulis swapped
    "commute-set-swapped": ("return softplus_neg(lam[t]) - log_sum_exp_neg(lam[u], lam[v]);",
                            "return softplus_neg(lam[u]) - log_sum_exp_neg(lam[t], lam[v]);"),
    # Eq. 3: tanh(|q|) instead of tanh(|q|/2)
    "bp-tanh-argument": ("prod *= tanh(0.5 * a);", "prod *= tanh(a);"),
    # Eqs. 3, 4, 8: the syndrome sign dropped
    "syndrome-sign-dropped": ("int neg = gbit(sy, i);", "int neg = 0;"),
    # Eqs. 4, 8: the check's own edge kept in the minimum
    "cn-not-extrinsic": ("if (f == e) continue;", "if (0) continue;"),
    # Eq. 7: eta on the input syndrome bit instead of the residual bit
    "eta-on-input-bit": ("(sres[i] ? eta_unsat : 1.0)", "(gbit(sy, i) ? eta_unsat : 1.0)"),
    # Eq. 6: the syndrome ratio over n
    "gamma-over-n": ("(double)unsat / (double)m", "(double)unsat / (double)n"),
    # Algorithm 1: ties of the Pauli decision resolved away from the identity
    "decision-ties": ("if (acc < best) { best = acc; arg = paulis[w]; }",
                      "if (acc <= best) { best = acc; arg = paulis[w]; }"),
    # Eq. 1: the residual from the commuting instead of the anticommuting estimates
    "residual-commuting": ("x ^= anticommute(ehat[col_idx[e]], pauli[e]);",
                           "x ^= (ehat[col_idx[e]] != 0) ^ anticommute(ehat[col_idx[e]], pauli[e]);"),
}


def _build(tmp_path, text):
    import oracle
    src = tmp_path / "gf4.c"
    src.write_text(text)
    lib = tmp_path / "libgf4_copy.so"
    subprocess.check_call(["gcc", *oracle.CFLAGS, str(src), "-o", str(lib), "-lm"])
    return str(lib)


def _run_pins(lib):
    env = {**os.environ, "ORACLE_GF4_LIB_OVERRIDE": lib}
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                           *PINS], capture_output=True, text=True, env=env, cwd=ROOT, timeout=900)


def _source():
    return open(os.path.join(ROOT, "oracle", "gf4.c")).read()


def test_unmodified_copy_passes_the_pins(tmp_path):
    r = _run_pins(_build(tmp_path, _source()))
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_fails_a_pin(tmp_path, name):
    old, new = MUTANTS[name]
    src = _source()
    assert src.count(old) == 1, f"{name}: the text to replace must occur exactly once in gf4.c"
    r = _run_pins(_build(tmp_path, src.replace(old, new)))
    assert r.returncode == 1 and " failed" in r.stdout, (name, r.returncode, r.stdout[-2000:])
