"""Planted mistakes in the oracle (CPU only).

Each mutant rewrites one spot of one oracle function with a plausible slip: a dropped term, a wrong
sign, index or operand, an off-by-one, a wrong constant.  The mutant runs in a fresh interpreter,
with the oracle's own pins (the tests that check it against the paper and the mathematics), and
at least one pin must fail.  This checks that the pins constrain the oracle.  It does not check the
oracle itself, and nothing here touches the CUDA library.

Mutation sites are plain text of the function's source; each must occur exactly once, so that a
later edit of the oracle that moves a site fails here loudly instead of testing nothing.
"""

import concurrent.futures
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

TENSOR = ["tests/test_oracle_tensor.py", "tests/test_oracle_tucker.py"]
RNG = ["tests/test_oracle_rng.py"]
STORAGE = ["tests/test_oracle_storage.py"]
TUCKER = ["tests/test_oracle_tucker.py", "tests/test_oracle_next.py"]
SELECT = ["tests/test_oracle_tucker.py", "tests/test_oracle_next.py", "tests/test_subset_select_cpu.py"]

# (id, module, function, text in the function, replacement, pin files)
MUTANTS = [
    # Sec. 2.1 tensor algebra
    ("unfold_column_order", "oracle.tensor", "unfold", 'order="F")', 'order="C")', TENSOR),
    ("fold_wrong_axis", "oracle.tensor", "fold", "np.moveaxis(T, 0, n)", "np.moveaxis(T, 0, -1)", TENSOR),
    ("ttm_transposed_operand", "oracle.tensor", "ttm", "fold(A @ unfold(X, n), n, shape)",
     "fold(A.T @ unfold(X, n), n, shape)", TENSOR),
    ("multi_ttm_ignores_transpose", "oracle.tensor", "multi_ttm", "M.T if transpose else M", "M", TENSOR),
    ("rel_error_squared_norm", "oracle.tensor", "rel_error", "/ frob(X)", "/ frob(X) ** 2", TENSOR),
    ("frob_drops_square_root", "oracle.tensor", "frob", "float(np.sqrt(", "float((", TENSOR),
    ("tucker_full_transposed_factors", "oracle.tensor", "tucker_full",
     "[np.asarray(A, dtype=np.float64) for A in factors]",
     "[np.asarray(A, dtype=np.float64)[::-1] for A in factors]", TENSOR),
    # Omega stream (Philox4x32-10, Box-Muller)
    ("philox_key_words_swapped", "oracle.rng", "philox4x32_10", "(hi1 ^ c1 ^ np.uint64(k0))",
     "(hi1 ^ c1 ^ np.uint64(k1))", RNG),
    ("philox_nine_rounds", "oracle.rng", "philox4x32_10", "range(10)", "range(9)", RNG),
    ("philox_weyl_constant", "oracle.rng", "philox4x32_10", "k1 = (k1 + W1)", "k1 = (k1 + W0)", RNG),
    ("uniform_not_odd", "oracle.rng", "uniform24", "| np.uint32(1)", "| np.uint32(0)", RNG),
    ("log_drops_series_term", "oracle.rng", "log_f32", "p = p * z + _L5", "p = p * z", RNG),
    ("log_series_doubling_dropped", "oracle.rng", "log_f32", "logm = (s + s) + t", "logm = s + t", RNG),
    ("log_exponent_not_bumped", "oracle.rng", "log_f32", "e = e + big.astype(np.int32)", "e = e", RNG),
    ("cossin_quadrant_sign", "oracle.rng", "cossin_2pi_f32", "[c, -s, -c], s)", "[c, s, -c], s)", RNG),
    ("sin_drops_series_term", "oracle.rng", "cossin_2pi_f32", "ps = ps * z + _S5", "ps = ps * z", RNG),
    ("box_muller_radius", "oracle.rng", "box_muller_f32", "F32(-2.0)", "F32(-1.0)", RNG),
    ("box_muller_words_swapped", "oracle.rng", "box_muller_f32", "cs, sn = cossin_2pi_f32(ub)",
     "cs, sn = cossin_2pi_f32(ua)", RNG),
    ("omega_counter_words_swapped", "oracle.rng", "omega", "q, dtype=np.uint64), lo, hi, sid",
     "q, dtype=np.uint64), hi, lo, sid", RNG),
    ("omega_column_order", "oracle.rng", "omega", "out[:, 4 * q + 1] = n1", "out[:, 4 * q + 1] = n2", RNG),
    ("bf16_ties_away", "oracle.rng", "round_bf16", "+ ((b >> np.uint64(16)) & np.uint64(1))", "+ np.uint64(1)",
     RNG),
    # E4M3 storage
    ("e4m3_bias", "oracle.storage", "e4m3_values", "2.0 ** (e - 7)", "2.0 ** (e - 8)", STORAGE),
    ("e4m3_subnormal_scale", "oracle.storage", "e4m3_values", "m * 2.0 ** -9", "m * 2.0 ** -10", STORAGE),
    ("fp8_scale_block", "oracle.storage", "fp8_dequantize", "np.arange(ld * mcols) // 128",
     "np.arange(ld * mcols) // 64", STORAGE),
    ("fp8_leading_dimension", "oracle.storage", "fp8_layout", "-(-dims[0] // 16) * 16", "dims[0]", STORAGE),
    # Alg. 1 (RandSVD) and Alg. 2 / 3
    ("randsvd_no_orthonormalisation", "oracle.tucker", "randsvd", "Q = canon_qr(Y)                                 #",
     "Q = Y                                 #", TUCKER),
    ("randsvd_factor_off_by_one", "oracle.tucker", "randsvd", "U = Q @ Ub[:, :r]", "U = Q @ Ub[:, 1:r + 1]", TUCKER),
    ("randsvd_power_step_missing", "oracle.tucker", "randsvd", "range(int(q))", "range(max(int(q) - 1, 0))",
     TUCKER),
    ("randsvd_extra_power_step", "oracle.tucker", "randsvd", "W = canon_qr(Xm.T @ Q)",
     "W = canon_qr(Xm.T @ canon_qr(Xm @ (Xm.T @ Q)))", TUCKER),
    ("sthosvd_reads_input", "oracle.tucker", "sthosvd", "_leading_left_sv(unfold(G, n)",
     "_leading_left_sv(unfold(X, n)", TUCKER),
    ("rhosvd_core_not_transposed", "oracle.tucker", "rhosvd", "multi_ttm(X, A, transpose=True)",
     "multi_ttm(X, A, transpose=False)", TUCKER),
    ("rsthosvd_core_drops_singular_values", "oracle.tucker", "rsthosvd", "fold(s[:, None] * V.T, n, shape)",
     "fold(V.T, n, shape)", TUCKER),
    ("rsthosvd_rank_off_by_one", "oracle.tucker", "rsthosvd", "r = min(int(ranks[n]), ell)",
     "r = min(int(ranks[n]), ell) - (1 if ranks[n] > 1 else 0)", TUCKER),
    ("rsthosvd_untruncated_drops_power_steps", "oracle.tucker", "rsthosvd", "Y = Gm @ canon_qr(Gm.T @ Q)",
     "Y = Y", TUCKER),
    # Sec. 4 (adaptive)
    ("adaptive_tail_off_by_one", "oracle.tucker", "adapt_range_finder", "np.sum(s[r:] ** 2) + res2",
     "np.sum(s[r + 1:] ** 2) + res2", TUCKER),
    ("adaptive_tail_drops_residual", "oracle.tucker", "adapt_range_finder", "np.sum(s[r:] ** 2) + res2",
     "np.sum(s[r:] ** 2)", TUCKER),
    ("adaptive_no_reorthogonalisation", "oracle.tucker", "adapt_range_finder", "Y = Y - Q @ (Q.T @ Y)", "Y = Y",
     TUCKER),
    ("adaptive_no_basis_completion", "oracle.tucker", "adapt_range_finder",
     "if np.abs(np.diag(Ri)).min() <= 1e-12 * gnorm:", "if False:", TUCKER),
    ("adaptive_tolerance_scaling", "oracle.tucker", "adaptive_rsthosvd", "/ math.sqrt(d)", "/ d", TUCKER),
    ("adaptive_rhosvd_tolerance_scaling", "oracle.tucker", "adaptive_rhosvd", "/ math.sqrt(d)", "/ d", TUCKER),
    # Sec. 5 (selections, SP-STHOSVD, SP-HOSVD, post-processing)
    ("srrqr_threshold", "oracle.tucker", "srrqr_select", "if amax <= eta:", "if amax <= 2.0 * eta:", SELECT),
    ("srrqr_no_swaps", "oracle.tucker", "srrqr_select", "for _ in range(max_swaps):", "for _ in range(0):",
     SELECT),
    ("deim_drops_absolute_value", "oracle.tucker", "deim_select", "np.argmax(np.abs(r))", "np.argmax(r)", SELECT),
    ("cpqr_takes_last_pivots", "oracle.tucker", "cpqr_select", "piv[:ell]", "piv[-ell:]", SELECT),
    ("leverage_weights_not_squared", "oracle.tucker", "sample_select",
     "s_ = s_ + float(Q[i, c]) * float(Q[i, c])", "s_ = s_ + abs(float(Q[i, c]))", SELECT),
    ("sp_sthosvd_factor_is_basis", "oracle.tucker", "sp_sthosvd", "A[n] = Q @ np.linalg.inv(Q[P, :])", "A[n] = Q",
     SELECT),
    ("sp_sthosvd_sketches_the_input", "oracle.tucker", "sp_sthosvd", "Y = unfold(G, n) @ Om",
     "Y = unfold(X, n)[:, :M] @ Om", SELECT),
    ("sp_hosvd_core_modes_reversed", "oracle.tucker", "sp_hosvd", "X[np.ix_(*sel)]",
     "np.transpose(X[np.ix_(*sel[::-1])], tuple(range(d))[::-1])", SELECT),
    ("kolda_rows_wrong_stride", "oracle.tucker", "_kolda_rows", "stride *= int(dims[k])", "stride *= int(dims[n])",
     SELECT),
    ("coo_sketch_drops_values", "oracle.tucker", "coo_sketch", "vals.astype(np.float64)[:, None] * om[inv]",
     "om[inv]", SELECT),
    ("coo_core_renumbering", "oracle.tucker", "sp_sthosvd_coo", "idx[:, n] = pos[idx[:, n]]",
     "idx[:, n] = pos[idx[:, n]][::-1]", SELECT),
    ("orthonormalize_transposed_triangle", "oracle.tucker", "orthonormalize_tucker", "G = ttm(G, R, n)",
     "G = ttm(G, R.T, n)", SELECT),
    # helpers shared by the algorithms
    ("default_order_increasing", "oracle.tucker", "default_order", "(-int(dims[n]), n)", "(int(dims[n]), n)",
     TUCKER),
    ("clamp_ignores_other_modes", "oracle.tucker", "_ell", "min(ell, int(I), int(M))", "min(ell, int(I))", TUCKER),
    ("strict_size_rule_lax", "oracle.tucker", "_check_ell", "ell < min(I, M) if strict", "ell <= min(I, M) if strict",
     TUCKER),
    ("canon_signs_flipped", "oracle.tucker", "canon_signs", "np.where(v < 0, -1.0, 1.0)", "np.where(v > 0, -1.0, 1.0)",
     TUCKER),
    ("omega_matrix_not_rounded", "oracle.tucker", "omega_matrix", 'if omega_round == "bf16":',
     'if omega_round == "never":', TUCKER),
    ("omega_matrix_wrong_mode", "oracle.tucker", "omega_matrix", "rng.omega(seed, tensor_id, mode,",
     "rng.omega(seed, tensor_id, 0,", TUCKER),
    ("coo_sketch_not_rounded", "oracle.tucker", "coo_sketch", 'if omega_round == "bf16":', 'if omega_round == "never":',
     SELECT),
    ("hosvd_rank_off_by_one", "oracle.tucker", "hosvd", "unfold(X, n), ranks[n])", "unfold(X, n), ranks[n] + 1)",
     TUCKER),
    ("uniform_sampling_stream_ignored", "oracle.tucker", "sample_select", "np.uint32(stream), np.uint32(0)",
     "np.uint32(0), np.uint32(0)", SELECT),
    ("sampling_keeps_taken_rows", "oracle.tucker", "sample_select", "taken[pick] = True", "taken[pick] = False",
     SELECT),
    ("sp_hosvd_selection_stream", "oracle.tucker", "sp_hosvd", "(int(tensor_id) << 4) | n)", "int(tensor_id) << 4)",
     SELECT),
    ("sp_coo_keeps_unselected", "oracle.tucker", "sp_sthosvd_coo", "keep = pos[idx[:, n]] >= 0",
     "keep = pos[idx[:, n]] >= -1", SELECT),
    ("fp8_rows_wrong_stride", "oracle.storage", "fp8_dequantize_rows", "e = int(i) + ld * p", "e = int(i) + dims[0] * p",
     STORAGE),
    ("omega_columns_wrong_lane", "oracle.rng", "omega_columns", "out[:, j] = groups[q][c % 4]",
     "out[:, j] = groups[q][(c + 1) % 4]", RNG),
    ("stream_id_shift", "oracle.rng", "stream_id", "(int(tensor_id) << 4) | int(mode)", "(int(tensor_id) << 3) | int(mode)",
     RNG),
    ("sp_bound_drops_growth", "oracle.tucker", "sp_bound", "gprod *= math.sqrt(1.0 + 4.0 * ell * (I - ell))",
     "gprod *= 1.0", TUCKER),
    ("sp_bound_growth_not_cumulative", "oracle.tucker", "sp_bound", "gprod *= math.sqrt(", "gprod = math.sqrt(", TUCKER),
    ("randsvd_v_signs_not_flipped", "oracle.tucker", "randsvd", "Vt[:r] *= sg[:, None]", "Vt[:r] *= 1.0", TUCKER),
    ("adaptive_omega_not_rounded", "oracle.tucker", "_omega_cols_fn", 'if omega_round == "bf16":',
     'if omega_round == "never":', TUCKER),
    ("sp_hosvd_coo_keeps_partial_matches", "oracle.tucker", "sp_hosvd_coo", "keep &= new[:, n] >= 0",
     "keep |= new[:, n] >= 0", SELECT),
    ("sp_hosvd_coo_sketches_renumbered", "oracle.tucker", "sp_hosvd_coo",
     "Y = coo_sketch(idx, vals, dims, n, ell,", "Y = coo_sketch(new, vals, dims, n, ell,", SELECT),
    ("e4m3_nan_code", "oracle.storage", "e4m3_values", "if e == 0xF and m == 0x7:", "if e == 0xF and m == 0x6:",
     STORAGE),
    # the error bounds of Sec. 3.2 / 5.2 (a bound that is too small fails the seed-averaged checks)
    ("bound_drops_one", "oracle.tucker", "randomized_bound", "(1.0 + ranks[n] / (p - 1.0))",
     "(ranks[n] / (p - 1.0))", TUCKER),
    ("delta_tail_off_by_one", "oracle.tucker", "delta2", "s[int(ranks[n]):]", "s[int(ranks[n]) + 1:]", TUCKER),
]

# Run by the fresh interpreter: apply one mutant to the oracle module (and to every oracle module
# that imported the function by name), then run the pin files; exit 7 if the mutant cannot be
# applied, else pytest's status (1 = some pin failed).
_DRIVER = r"""
import importlib, inspect, sys, textwrap
mod_name, func, old, new = sys.argv[1:5]
pins = sys.argv[5:]
try:
    mod = importlib.import_module(mod_name)
    orig = getattr(mod, func)
    src = textwrap.dedent(inspect.getsource(orig))
    if src.count(old) != 1:
        raise RuntimeError(f"mutation site found {src.count(old)} times in {mod_name}.{func}")
    exec(compile(src.replace(old, new), mod.__file__, "exec"), mod.__dict__)
    mutant = getattr(mod, func)
    if mutant is orig:
        raise RuntimeError("the mutant did not replace the function")
    for name, m in list(sys.modules.items()):
        if name == "oracle" or name.startswith("oracle."):
            for attr, val in list(vars(m).items()):
                if val is orig:
                    setattr(m, attr, mutant)
except Exception as e:
    print("MUTANT NOT APPLIED:", repr(e))
    sys.exit(7)
import pytest
sys.exit(pytest.main(["-x", "-q", "-rf", "-p", "no:cacheprovider", "-m", "not gpu", *pins]))
"""


# one BLAS thread per interpreter: the mutants run side by side
_ENV = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


def _run(m):
    mid, module, func, old, new, pins = m
    try:
        r = subprocess.run([sys.executable, "-c", _DRIVER, module, func, old, new, *pins], cwd=ROOT,
                           capture_output=True, text=True, timeout=300, env=_ENV)
        return mid, r.returncode, (r.stdout + r.stderr)[-3000:]
    except subprocess.TimeoutExpired:
        return mid, -1, "timed out"


@pytest.fixture(scope="module")
def outcomes(request):
    # the mutants of the selected tests, run side by side (each in its own interpreter)
    wanted = {it.callspec.params["mid"] for it in request.session.items
              if hasattr(it, "callspec") and "mid" in it.callspec.params}
    todo = [m for m in MUTANTS if m[0] in wanted]
    workers = max(1, min(8, os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        return {mid: (rc, out) for mid, rc, out in ex.map(_run, todo)}


def test_mutant_ids_are_unique():
    ids = [m[0] for m in MUTANTS]
    assert len(ids) == len(set(ids))


@pytest.mark.parametrize("mid", [m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(outcomes, mid):
    rc, out = outcomes[mid]
    assert rc != 7, out                      # the mutation site must exist exactly once
    assert rc == 1, f"mutant {mid} survived the pins (pytest status {rc}):\n{out}"
