"""Planted mistakes in the oracle are caught by its pins.

Each case copies ``oracle/`` and the seeded input generator into a scratch
directory, plants one plausible mistake in the copy by an exact text
substitution (a dropped term, a wrong sign or index, a transposed operand, a
swapped convention), and runs the oracle's pin tests (tests/test_oracle.py,
tests/test_oracle_distinguishable.py) against the copy in a child process: at
least one pin must fail, while the unchanged copy passes them all.  The copy
builds its own C library; the repository's files are not modified.  A case
whose text no longer occurs exactly once fails loudly, so the list follows the
oracle's source.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = [os.path.join(ROOT, "tests", f) for f in ("test_oracle.py", "test_oracle_distinguishable.py")]

# files of the scratch copy: the oracle package and the seeded input generator
C, PY, DIST, MLP = "oracle/pcv_oracle.c", "oracle/__init__.py", "oracle/distinguishable.py", "oracle/mlp.py"
INPUTS = "pcv_inputs.py"

# (name, file, text, replacement)
MUTATIONS = [
    # Ryser's formula
    ("ryser_sign_dropped", C, "if (((n - size) & 1) != 0) prod = -prod;", ";"),
    ("ryser_sign_parity_of_size", C, "if (((n - size) & 1) != 0) prod = -prod;",
     "if ((size & 1) != 0) prod = -prod;"),
    ("ryser_gray_update_transposed", C,
     "if (gk & (1ull << j)) for (int i = 0; i < n; ++i) rs[i] += A[i * n + j];",
     "if (gk & (1ull << j)) for (int i = 0; i < n; ++i) rs[i] += A[j * n + i];"),
    ("ryser_gray_removal_adds", C,
     "else                  for (int i = 0; i < n; ++i) rs[i] -= A[i * n + j];",
     "else                  for (int i = 0; i < n; ++i) rs[i] += A[i * n + j];"),
    ("ryser_block_start_not_gray", C, "cplx rs[64];\n    uint64_t g = k0 ^ (k0 >> 1);",
     "cplx rs[64];\n    uint64_t g = k0;"),
    ("ryser_last_block_dropped", C, "for (int64_t b = 0; b < nblocks; ++b) { nsum_add(&re, creal(part[b]));",
     "for (int64_t b = 0; b + 1 < nblocks; ++b) { nsum_add(&re, creal(part[b]));"),
    # the definition
    ("leibniz_sum_not_product", C, "prefix * A[row * n + j]", "prefix + A[row * n + j]"),
    ("leibniz_columns_reused", C, "if (!(used & (1ull << j)))", "if (row >= 0)"),
    # double-double arithmetic
    ("dd_two_sum_error_dropped", C, "double e = (a - (s - bb)) + (b - bb);", "double e = 0.0;"),
    ("dd_product_remainder_dropped", C, "double e = fma(a.hi, b.hi, -p);", "double e = 0.0;"),
    ("dd_complex_product_sign", C, "{dd_add(dd_mul(a.re, b.re), dd_neg(dd_mul(a.im, b.im))),",
     "{dd_add(dd_mul(a.re, b.re), dd_mul(a.im, b.im)),"),
    # Eq. eqperm: submatrix and normalisation
    ("submatrix_rows_by_input", C, "A[a * nr + b] = U[(size_t)rows[a] * m + cols[b]];",
     "A[a * nr + b] = U[(size_t)cols[b] * m + rows[a]];"),
    ("norm_without_input_factorials", C, "d *= factorial(out_occ[i]) * factorial(in_occ[i]);",
     "d *= factorial(out_occ[i]);"),
    ("norm_without_square_root", C, "return 1.0 / sqrt(d);", "return 1.0 / d;"),
    ("factorial_one_factor_short", C, "for (int i = 2; i <= k; ++i) f *= (double)i;",
     "for (int i = 2; i < k; ++i) f *= (double)i;"),
    ("photon_number_not_checked", C, "if (nr != nc || nr > 40) return -1;", "if (nr > 40 || nc > 40) return -1;"),
    # output space
    ("num_outputs_binomial_shifted", C, "c = c * (unsigned __int128)(m - 1 + k) / (unsigned __int128)k;",
     "c = c * (unsigned __int128)(m + k) / (unsigned __int128)k;"),
    ("enumerate_last_photon_dropped", C, "for (int i = 0; i < n; ++i) o[modes[i]]++;",
     "for (int i = 0; i + 1 < n; ++i) o[modes[i]]++;"),
    ("probability_real_part_only", C, "prob[o] = a[0] * a[0] + a[1] * a[1];", "prob[o] = a[0] * a[0];"),
    # Laplace gradient
    ("grad_minor_wrong_column", C, "if (b == j) continue;", "if (b == i) continue;"),
    ("grad_scatter_transposed", C, "D[(size_t)rows[i] * m + cols[j]] +=", "D[(size_t)cols[j] * m + rows[i]] +="),
    ("grad_without_normalisation", C, "+= (p[0] + I * p[1]) * nrm;", "+= (p[0] + I * p[1]);"),
    ("grad_convention_without_conjugate", PY, "G += g * np.conj(amplitude_grad(U, input_occ, s))",
     "G += g * amplitude_grad(U, input_occ, s)"),
    # mesh (Eq. bs, MZI, Clements layout)
    ("mesh_composition_reversed", PY, "        U = T @ U", "        U = U @ T"),
    ("clements_column_parity_swapped", PY, "for k in range(c % 2, m - 1, 2):", "for k in range(1 - c % 2, m - 1, 2):"),
    ("mzi_inner_phase_on_lower_mode", PY, "ps_a = np.diag([np.exp(1j * phi_a), 1.0])",
     "ps_a = np.diag([1.0, np.exp(1j * phi_a)])"),
    ("mzi_outer_phase_first", PY, "return ps_b @ BS_RX_HALF @ ps_a @ BS_RX_HALF",
     "return BS_RX_HALF @ ps_a @ BS_RX_HALF @ ps_b"),
    ("beam_splitter_conjugate_convention", PY, "[[1.0, 1.0j], [1.0j, 1.0]]", "[[1.0, -1.0j], [-1.0j, 1.0]]"),
    # distances
    ("tvd_without_half", PY, "return 0.5 * float(", "return float("),
    ("kl_direction_reversed", PY, "return float(np.sum(q[nz] * (np.log(q[nz]) - np.log(p[nz]))))",
     "return float(np.sum(p[p > 0] * (np.log(p[p > 0]) - np.log(q[p > 0]))))"),
    # photon classes and sources
    ("source_weights_swapped", DIST, "w = q ** (n - size) * (1.0 - q) ** size", "w = q ** size * (1.0 - q) ** (n - size)"),
    ("class_convolution_overwrites", DIST, "new_p[idx[summed[b].astype(np.uint8).tobytes()]] += cur_p[a] * p_g[b]",
     "new_p[idx[summed[b].astype(np.uint8).tobytes()]] = cur_p[a] * p_g[b]"),
    ("lossy_pure_and_noisy_swapped", DIST, "(eta * q if st == 1 else eta * (1.0 - q))",
     "(eta * (1.0 - q) if st == 1 else eta * q)"),
    ("noisy_photons_share_one_class", DIST, "            out.append(t)\n",
     "            out = [out[0] + t] if out else [t]\n"),
    # surrogate network reference
    ("bf16_truncates", MLP, "u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000", "u = u & 0xFFFF0000"),
    ("bf16_ties_away_from_zero", MLP, "u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000", "u = (u + 0x8000) & 0xFFFF0000"),
    ("gelu_wrong_scale", MLP, "return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))", "return 0.5 * x * (1.0 + erf(x / 2.0))"),
    ("gelu_grad_term_dropped", MLP, " + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)", ""),
    ("adam_without_bias_correction", MLP, "(m / (1 - b1 ** step))", "m"),
    ("adam_eps_inside_root", MLP, "(np.sqrt(v / (1 - b2 ** step)) + eps)", "np.sqrt(v / (1 - b2 ** step) + eps)"),
    ("mse_gradient_without_factor_two", MLP, "2.0 * d / d.size", "d / d.size"),
    ("features_without_constant", MLP, "    X[:, 2 * P] = 1.0\n", ""),
    ("forward_bias_dropped", MLP, "pre = gemm(h, W) + b", "pre = gemm(h, W)"),
    ("forward_hidden_layer_linear", MLP, "h = bf16(gelu(pre))", "h = bf16(pre)"),
    # the Haar unitaries both sides are fed
    ("haar_without_phase_fix", INPUTS, "return np.ascontiguousarray(q * ph[None, :], dtype=np.complex128)",
     "return np.ascontiguousarray(q, dtype=np.complex128)"),
    ("haar_from_real_gaussians", INPUTS,
     "z = (g.standard_normal((m, m)) + 1j * g.standard_normal((m, m))) / np.sqrt(2.0)\n    q, r",
     "z = g.standard_normal((m, m)) + 0j\n    q, r"),
]


def child_env(scratch, threads=1):
    env = dict(os.environ)
    env["PYTHONPATH"] = os.pathsep.join([str(scratch), ROOT] + ([env["PYTHONPATH"]] if env.get("PYTHONPATH") else []))
    env["OMP_NUM_THREADS"] = str(threads)          # the cases run side by side
    return env


def run_pins(scratch, env, extra):
    return subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider",
                           "--basetemp", str(scratch / "pins"), *extra],
                          cwd=str(scratch), env=env, capture_output=True, text=True, timeout=1800)


QUICK = ["-m", "not gpu and not slow", "-k", "not under_cancellation"]
FULL = ["-m", "not gpu"]


def plant(scratch, name, fname, text, repl):
    """(phase that caught the mistake: 0 quick pins, 1 all pins; or None, why not)."""
    scratch.mkdir()
    copy = scratch / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), copy, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copy(os.path.join(ROOT, INPUTS), scratch / INPUTS)
    if fname is not None:
        src = (scratch / fname).read_text()
        if src.count(text) != 1:
            return None, f"{name}: the text to change occurs {src.count(text)} times in {fname}"
        (scratch / fname).write_text(src.replace(text, repl))
    # the unchanged copy runs every pin, the longest case: give it more threads
    env = child_env(scratch, 1 if fname is not None else max(1, (os.cpu_count() or 2) // 2))
    # the child imports the copy, and the copy builds
    probe = subprocess.run([sys.executable, "-c", "import oracle, pcv_inputs; oracle.build(); "
                            "print(oracle.__file__); print(pcv_inputs.__file__)"],
                           cwd=str(scratch), env=env, capture_output=True, text=True, timeout=300)
    if probe.returncode != 0 or not all(f.startswith(str(scratch)) for f in probe.stdout.split()):
        return None, f"{name}: the copy did not load: {probe.stdout[-300:]} {probe.stderr[-1500:]}"
    # the quick pins first; all of them only when those pass
    for phase, extra in enumerate((QUICK, FULL)):
        r = run_pins(scratch, env, extra)
        if r.returncode == 1:              # tests ran and one failed: caught
            return phase, ""
        if r.returncode != 0:
            return None, f"{name}: the pins did not run (exit {r.returncode}): {r.stdout[-1500:]}"
    return None, f"{name} survived the pins:\n{r.stdout[-500:]}"


def test_every_planted_mistake_fails_a_pin(tmp_path):
    workers = max(1, min(8, os.cpu_count() or 1))
    cases = [("unchanged", None, None, None)] + MUTATIONS
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda case: plant(tmp_path / case[0], *case), cases))
    # control: the unchanged copy passes every pin in the same setting
    (phase, why), results = results[0], results[1:]
    assert phase is None and why.startswith("unchanged survived"), why
    failures = [why for phase, why in results if phase is None]
    assert not failures, "\n\n".join(failures)
