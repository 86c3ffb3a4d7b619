"""The oracle's pins catch plausible mistakes (CPU).

Each case plants one mistake in a copy of oracle/oracle.c (the oracle itself is never
modified), compiles the copy with the oracle's own flags, and runs the pin files against it
in a subprocess (ORACLE_LIB_OVERRIDE points the oracle package at the copy).  At least one
pin must fail.  A control run of the unmodified copy, built the same way, must pass, so a
failure is the pins' doing and not the harness's.

One plausible mistake is left out because it is equivalent, not missed: taking sgn(0) = -1
for a zero incoming message in the sign product.  A zero input makes every other edge's
output magnitude zero (the MS minimum, or the BP tanh product), so its sign never reaches a
posterior and no decision or count can show it."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = [os.path.join(ROOT, "tests", "test_oracle_pins.py")]
LAYERED_PINS = [os.path.join(ROOT, "tests", "test_layered_oracle.py")]
AUTO_PINS = [os.path.join(ROOT, "tests", "test_auto_ceiling.py")]

# name: (text in oracle.c, replacement, pin files that must catch it)
MUTANTS = {
    # Eq. 7: the eta boost on the input syndrome bit instead of the residual bit
    "eta-on-input-bit": ("eta_unsat, gamma, sres[i]);", "eta_unsat, gamma, bit_of(sy, i));", PINS),
    # Eq. 6: the syndrome ratio over the qubits instead of the checks
    "gamma-over-n": ("syndrome_ratio(unsat, m)", "syndrome_ratio(unsat, n)", PINS),
    # Eq. 7: the gain schedule inverted (rising with the unsatisfied fraction)
    "gain-schedule-inverted": ("(amax - (amax - alpha_min) * gamma)", "(alpha_min + (amax - alpha_min) * gamma)",
                               PINS),
    # Eqs. 3, 4, 8: the (-1)^{s_i} factor dropped
    "syndrome-sign-dropped": ("int sg = s_i;", "int sg = 0;", PINS),
    # Eqs. 4, 8: the check's own edge kept in the minimum (not extrinsic)
    "cn-not-extrinsic": ("if (f == e) continue;", "if (0) continue;", PINS),
    # Eq. 3: tanh(|q|) instead of tanh(|q| / 2)
    "bp-tanh-argument": ("pr *= tanh(0.5 * a);", "pr *= tanh(a);", PINS),
    # Eq. 3: atanh without its factor 2
    "bp-atanh-factor": ("2.0 * atanh(prod)", "atanh(prod)", PINS),
    # Eq. 2: the VN->CN message includes the receiving check's own message (not extrinsic)
    "vn-not-extrinsic": ("                            if (u != t) {", "                            if (1) {", PINS),
    # Eq. 2: the prior left out of the VN->CN message
    "vn-prior-dropped": ("double acc = prior[j], mag = fabs(prior[j]);\n                        for (int u = vn_ptr[j]; "
                         "u < vn_ptr[j + 1]; ++u)\n                            if (u != t) {",
                         "double acc = 0.0, mag = fabs(prior[j]);\n                        for (int u = vn_ptr[j]; "
                         "u < vn_ptr[j + 1]; ++u)\n                            if (u != t) {", PINS),
    # Algorithm 1: iterations counted one too many at the early exit
    "iters-off-by-one": ("conv[s] = 1; iters[s] = l; break;", "conv[s] = 1; iters[s] = l + 1; break;", PINS),
    # Eq. 1: the residual ignores the input syndrome
    "residual-without-syndrome": ("int x = bit_of(sy, i);\n                for (int e", "int x = 0;\n                for (int e",
                                  PINS),
    # layered schedule: each check's inputs from the round's start, not the messages as they stand
    "layered-stale-inputs": ("                    cn_update(i, row_ptr, bit_of(sy, i), msfam, gain[i], q, r, &nclip);\n"
                             "                }\n            }",
                             "                }\n                for (int o = 0; o < m; ++o) {\n"
                             "                    const int i = order[o];\n"
                             "                    cn_update(i, row_ptr, bit_of(sy, i), msfam, gain[i], q, r, &nclip);\n"
                             "                }\n            }", LAYERED_PINS),
    # reading 1: a posterior of exactly zero decided as a flip
    "decision-tie": ("ehat[j] = (acc < 0.0) ? 1 : 0;", "ehat[j] = (acc <= 0.0) ? 1 : 0;", PINS),
    # reading 3: negative per-shot priors lose their sign in L0-normalised units
    "normalised-prior-sign": ("if (normalise) l0 = (l0 > 0.0) ? 1.0 : ((l0 < 0.0) ? -1.0 : 0.0);",
                              "if (normalise) l0 = 1.0;", PINS),
    # reading 8: the clips changed
    "msfam-clip": ("static const double MSFAM_CLIP = 1.0e6;", "static const double MSFAM_CLIP = 1.0e5;", PINS),
    "bp-clip": ("static const double BP_CLIP = 23.718998;", "static const double BP_CLIP = 20.0;", PINS),
    # reading 10: a non-finite prior decoded instead of marking the shot invalid
    "invalid-prior-ignored": ("if (!isfinite(per_qubit ? L0[j] : L0[s])) bad = 1;", "", PINS),
    # per-qubit priors read from the wrong qubit
    "per-qubit-index": ("prior_in_units(per_qubit ? L0[j] : L0[s],", "prior_in_units(per_qubit ? L0[0] : L0[s],", PINS),
    # Algorithm 1: early stop taken although SAGMS_FLAG_NO_EARLY_STOP is set
    "no-early-stop-ignored": ("if (unsat == 0 && early_stop)", "if (unsat == 0)", PINS),
    # Algorithm 1: a zero residual at the last round reported as not converged
    "conv-at-max-iter": ("conv[s] = (unsat == 0); iters[s] = max_iter;", "conv[s] = 0; iters[s] = max_iter;", PINS),
    # Corollary 1: the automatic ceiling without its clamp to [alpha_min, 1/eta]
    "auto-ceiling-no-upper-clamp": ("if (a > 1.0 / eta_unsat) a = 1.0 / eta_unsat;", "", AUTO_PINS),
    "auto-ceiling-no-lower-clamp": ("if (!(a >= alpha_min)) a = alpha_min;", "", AUTO_PINS),
    # layered schedule: checks visited in index order, not layer order
    "layered-index-order": ("            if (layer[i] == l) order[o++] = i;",
                            "            if (layer[i] == l) { order[o] = o; ++o; }", LAYERED_PINS),
    # layered schedule: a check's input includes its own old message
    "layered-vn-not-extrinsic": ("                            if (vn_edges[u] != e) {",
                                 "                            if (1) {", LAYERED_PINS),
    # layered schedule: layers that are valid but not first-fit (odd checks one layer up)
    "layered-not-first-fit": ("while (stamp[l]) ++l;", "while (stamp[l]) ++l; l = (i % 2) ? l + 1 : l;", LAYERED_PINS),
}


def _build(tmp_path, text):
    import oracle
    src = tmp_path / "oracle.c"
    src.write_text(text)
    lib = tmp_path / "liboracle_copy.so"
    subprocess.check_call(["gcc", *oracle.CFLAGS, str(src), "-o", str(lib), "-lm"])
    return str(lib)


def _run_pins(lib, files):
    env = {**os.environ, "ORACLE_LIB_OVERRIDE": lib}
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                           *files], capture_output=True, text=True, env=env, cwd=ROOT, timeout=900)


def _source():
    return open(os.path.join(ROOT, "oracle", "oracle.c")).read()


def test_unmodified_copy_passes_the_pins(tmp_path):
    r = _run_pins(_build(tmp_path, _source()), PINS + LAYERED_PINS + AUTO_PINS)
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_fails_a_pin(tmp_path, name):
    old, new, files = MUTANTS[name]
    src = _source()
    assert src.count(old) == 1, f"{name}: the text to replace must occur exactly once in oracle.c"
    r = _run_pins(_build(tmp_path, src.replace(old, new)), files)
    # exit code 1: a test failed (not a crash, a collection error or an interrupted run)
    assert r.returncode == 1 and " failed" in r.stdout, (name, r.returncode, r.stdout[-2000:])
