"""Planted mistakes: every pin-guarded slip in the FP64 oracle is caught by a pin.

Each case below rewrites one expression of ``oracle/oracle.cpp`` into a plausible
mistake (a dropped term, a wrong sign, a missing conjugate, a transposed operand, a
wrong threshold or an off-by-one layer index), compiles the result into a separate
library under the test's temporary directory, and runs the pins of
``test_oracle_pins.py`` against it in a child process, cheapest first, until one
fails.  The case passes when some pin fails.  The unmodified source compiled the
same way passes every pin (the control case), so a failure is the planted
mistake's doing.  The oracle's own library and source are never touched.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.cpp")

# (case, exact text in oracle.cpp, replacement)
PLANTED = [
    ("residual drops S", "      if (k == j) s -= t[k];\n", ""),
    ("residual conjugates H", "s += W[k * M + m] * H[j * M + m];",
     "s += W[k * M + m] * std::conj(H[j * M + m]);"),
    ("Gram transposed", "s += H[k * M + m] * std::conj(H[j * M + m]);",
     "s += std::conj(H[k * M + m]) * H[j * M + m];"),
    ("prox factor sign", "(r > tau) ? (1.0 - tau / r) : 0.0", "(r > tau) ? (1.0 + tau / r) : 0.0"),
    ("prox on squared norm", "    const double r = std::sqrt(p);\n    const double f = (r > tau)",
     "    const double r = p;\n    const double f = (r > tau)"),
    ("update without conj(H)", "s += Y[k * K + j] * std::conj(H[j * M + m]);",
     "s += Y[k * K + j] * H[j * M + m];"),
    ("update sign", "W[k * M + m] -= scale * s;", "W[k * M + m] += scale * s;"),
    ("ZF without conjugate", "W[k * M + m] = t[k] * std::conj(x[k]);", "W[k * M + m] = t[k] * x[k];"),
    ("paper-layer threshold without eta", "prox_l21(K, M, W, lam * eta);", "prox_l21(K, M, W, lam);"),
    ("paper-layer start H instead of H^*", "W[i] = std::conj(H[i]);  // W^(0) = H^*",
     "W[i] = H[i];  // W^(0) = H^*"),
    ("projected layer projects before shrinking",
     "    prox_l21(K, M, W, mu[l]);\n    project_affine(K, M, H, t, L.data(), W);\n",
     "    project_affine(K, M, H, t, L.data(), W);\n    prox_l21(K, M, W, mu[l]);\n"),
    ("Cholesky without conjugate", "s -= L[i * K + p] * std::conj(L[j * K + p]);",
     "s -= L[i * K + p] * L[j * K + p];"),
    ("back substitution without conjugate", "s -= std::conj(L[p * K + i]) * x[p];",
     "s -= L[p * K + i] * x[p];"),
    ("l2,1 without square root", "    s += std::sqrt(p);\n", "    s += p;\n"),
    ("ADMM dual update sign", "U[i] += W[i] - Z[i];", "U[i] += Z[i] - W[i];"),
    ("ADMM threshold rho instead of 1/rho", "prox_l21(K, M, Z.data(), 1.0 / rho);",
     "prox_l21(K, M, Z.data(), rho);"),
    ("shrink adjoint sign", "c2 = tau / (r * r * r) * vg;", "c2 = -tau / (r * r * r) * vg;"),
    ("loss gradient without factor 2", "G[k * M + m] = 2.0 * s;", "G[k * M + m] = s;"),
    ("supervised gradient without factor 2", "      G[i] = 2.0 * d;", "      G[i] = d;"),
    ("supervised gradient with the label's sign", "      const cd d = W[i] - Wgt[i];",
     "      const cd d = W[i] + Wgt[i];"),
    ("paper-layer d/deta drops the threshold term", "deta[l] = -gv_eh + lam[l] * dtau;",
     "deta[l] = -gv_eh;"),
    ("projected-layer adjoint one layer off",
     "dmu[l] = shrink_backward(K, M, trace.data() + (size_t)l * n,",
     "dmu[l] = shrink_backward(K, M, trace.data() + (size_t)(l + 1) * n,"),
    ("SINR noise as amplitude", "sinr[k] = sig / (intf + sigma * sigma);",
     "sinr[k] = sig / (intf + sigma);"),
    ("sum rate in nats", "r += std::log2(1.0 + s[k]);", "r += std::log(1.0 + s[k]);"),
    ("PCG inverted", "return l21(K, M, Wz.data()) / l21(K, M, as_c(W));",
     "return l21(K, M, as_c(W)) / l21(K, M, Wz.data());"),
    ("penalised objective without factor 2", "return 2.0 * lam * l21(K, M, as_c(W)) + fro2",
     "return lam * l21(K, M, as_c(W)) + fro2"),
    ("batch harness swaps eta and lambda",
     "orc_ufpgd_forward(K, M, Hb, tb, T, p1, p2, nullptr, Wb, nullptr)",
     "orc_ufpgd_forward(K, M, Hb, tb, T, p2, p1, nullptr, Wb, nullptr)"),
    ("batch harness drops the last instance of a range",
     "long b0 = i * per, b1 = std::min(B, b0 + per);\n    if (b0 >= b1) break;\n"
     "    th.emplace_back(work, b0, b1);\n  }\n  for (auto& x : th) x.join();\n  return ORC_OK;\n}\n\n"
     "// Same split",
     "long b0 = i * per, b1 = std::min(B, b0 + per - 1);\n    if (b0 >= b1) break;\n"
     "    th.emplace_back(work, b0, b1);\n  }\n  for (auto& x : th) x.join();\n  return ORC_OK;\n}\n\n"
     "// Same split"),
    ("power iteration normalised by sqrt", "for (int i = 0; i < K; ++i) v[i] = w[i] / nw;",
     "for (int i = 0; i < K; ++i) v[i] = w[i] / std::sqrt(nw);"),
]

# Cheapest pins first; the long-run solves come last.
ORDER = [
    ("test_l21_and_residual_definitions", {}),
    ("test_gram_cholesky_and_singular", {}),
    ("test_zf_matches_svd_pseudoinverse", {}),
    ("test_pcg_definition", {}),
    ("test_projection_idempotent_and_feasible", {}),
    ("test_projected_layers_feasible_every_layer", {}),
    ("test_paper_layer_one_step_and_lambda_zero_limit", {}),
    ("test_paper_layer_monotone_descent", {}),
    ("test_batch_forward_matches_single_instances", {}),
    ("test_prox_l21_is_the_proximal_map", {}),
    ("test_projected_layer_gradient_vs_central_differences", {}),
    ("test_paper_layer_gradient_vs_central_differences", {}),
    ("test_supervised_loss_gradients", {}),
    ("test_square_channel_leaves_no_freedom", {}),
    ("test_feasible_precoder_hits_paper_sum_rate", {}),
    ("test_single_user_penalised_closed_form_and_factor_two", {}),
    ("test_penalised_brute_force", {}),
    ("test_single_user_constrained_closed_form", {}),
    ("test_diminishing_projected_layers_approach_the_admm_optimum", {}),
    ("test_admm_kkt_certificate", {}),
    ("test_constrained_brute_force", dict(K=1, M=2, seed=8)),
    ("test_constrained_brute_force", dict(K=2, M=3, seed=9)),
    ("test_constrained_brute_force", dict(K=1, M=3, seed=10)),
    ("test_constrained_optimum_reproduces_paper_pcg", {}),
]

# Child process: load the given library in place of the oracle's own and run the
# pins in ORDER; print the first pin that fails (or "none") and exit.
_RUNNER = r"""
import ctypes, json, sys
sys.path.insert(0, sys.argv[2]); sys.path.insert(0, sys.argv[3])
import oracle
lib = ctypes.CDLL(sys.argv[1])
oracle._declare(lib)
oracle._lib = lib
import test_oracle_pins as pins
for name, kw in json.loads(sys.argv[4]):
    try:
        getattr(pins, name)(oracle, **kw)
    except Exception as e:
        print("CAUGHT", name, type(e).__name__, flush=True)
        sys.exit(0)
print("CAUGHT none", flush=True)
"""


def _compile(src_text, out_dir):
    cpp = os.path.join(out_dir, "oracle_planted.cpp")
    so = os.path.join(out_dir, "liboracle_planted.so")
    with open(cpp, "w") as f:
        f.write(src_text)
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fPIC", "-shared",
                           "-pthread", cpp, "-o", so])
    return so


def _first_failing_pin(so, timeout):
    import json
    r = subprocess.run([sys.executable, "-c", _RUNNER, so, ROOT, os.path.join(ROOT, "tests"),
                        json.dumps(ORDER)], capture_output=True, text=True, timeout=timeout)
    lines = [l for l in r.stdout.splitlines() if l.startswith("CAUGHT ")]
    assert r.returncode == 0 and lines, (r.returncode, r.stdout[-2000:], r.stderr[-2000:])
    return lines[-1].split()[1]


def test_unmodified_source_passes_every_pin(tmp_path):
    with open(SRC) as f:
        src = f.read()
    assert _first_failing_pin(_compile(src, str(tmp_path)), timeout=600) == "none"


@pytest.mark.parametrize("case,old,new", PLANTED, ids=[p[0] for p in PLANTED])
def test_planted_mistake_is_caught(tmp_path, case, old, new):
    with open(SRC) as f:
        src = f.read()
    assert src.count(old) == 1, f"the text to plant '{case}' in must occur exactly once"
    caught = _first_failing_pin(_compile(src.replace(old, new), str(tmp_path)), timeout=600)
    assert caught != "none", f"no pin fails with '{case}' planted"


def test_order_lists_every_pin():
    """Every pin of test_oracle_pins.py takes part in the planted-mistake runs."""
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import test_oracle_pins as pins
    names = {n for n in dir(pins) if n.startswith("test_")}
    assert names == {n for n, _ in ORDER}
