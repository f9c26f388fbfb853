"""ctypes binding of libpcv.so (declarations in include/pcv.h).

The functions named pcv_* take exactly the C arguments (device pointers may
be given as torch tensors) and raise PcvError on a negative return code.
There is no fallback: if libpcv.so is missing this module raises on import.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpcv.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -m paper_2204_00602_gb300.build)")

_lib = ctypes.CDLL(LIB_PATH)

PCV_OK = 0
PCV_EINVAL = -1
PCV_ERANGE = -2
PCV_ECUDA = -3
PCV_ETIMEOUT = -4
PCV_ENOMEM = -5
PCV_ALGO_AUTO = 0
PCV_ALGO_GROUP = 1
PCV_ALGO_BLOCK = 2
PCV_ALGO_FACTOR = 3
PCV_ALGO_TILE = 4
PCV_ALGO_SLOS = 5
PCV_ALGO_MULT = 6
PCV_ALGO_FACTOR_TC = 7
PCV_MAX_PHOTONS = 30
PCV_MAX_MODES = 1024

_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64

# name -> (restype, argtypes); every symbol include/pcv.h declares
SIGNATURES = {
    "pcv_last_error": (ctypes.c_char_p, []),
    "pcv_version": (ctypes.c_char_p, []),
    "pcv_num_outputs": (_i64, [_i, _i]),
    "pcv_unrank": (_i, [_i, _i, _i64, _vp]),
    "pcv_rank": (_i64, [_i, _vp]),
    "pcv_amplitudes_workspace": (_i64, [_i, _i, _i64]),
    "pcv_amplitudes": (_i, [_vp, _i, _vp, _vp, _i64, _vp, _vp, _vp, _i64, _vp]),
    "pcv_amplitudes_ex": (_i, [_vp, _i, _vp, _vp, _i64, _vp, _vp, _i, _i, _vp, _i64, _vp]),
    "pcv_amplitudes_ex_workspace": (_i64, [_i, _i, _i64, _i, _i]),
    "pcv_distribution_workspace": (_i64, [_i, _i]),
    "pcv_distribution_tc_workspace": (_i64, [_i, _i]),
    "pcv_distribution_workspace_min": (_i64, [_i, _i]),
    "pcv_distribution_auto_algo": (_i, [_i, _i, _i64]),
    "pcv_distribution": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _i64, _vp]),
    "pcv_distribution_ex": (_i, [_vp, _i, _vp, _vp, _vp, _i, _i, _vp, _i64, _vp]),
    "pcv_distribution_range": (_i, [_vp, _i, _vp, _i64, _i64, _vp, _vp, _vp, _i64, _vp]),
    "pcv_distribution_range_plan": (_i, [_i, _i, _i64, _i64, _vp, _vp]),
    "pcv_distribution_tc_blocks": (_i, [_i, _i, _i64, _i64, _vp, _i64, _vp]),
    "pcv_distribution_batched_workspace": (_i64, [_i, _i, _i]),
    "pcv_distribution_batched": (_i, [_vp, _i, _i, _vp, _vp, _vp, _vp, _i64, _vp]),
    "pcv_distribution_slos_workspace": (_i64, [_i, _i, _i]),
    "pcv_distribution_slos": (_i, [_vp, _i, _i, _vp, _vp, _vp, _vp, _i64, _vp]),
    "pcv_amplitudes_backward_workspace": (_i64, [_i, _i, _i, _i64]),
    "pcv_amplitudes_backward": (_i, [_vp, _i, _vp, _vp, _i64, _vp, _vp, _vp, _i64, _vp]),
    "pcv_distribution_backward_workspace": (_i64, [_i, _i, _i]),
    "pcv_distribution_backward": (_i, [_vp, _i, _i, _vp, _vp, _vp, _vp, _i64, _vp]),
    "pcv_mesh_unitary": (_i, [_vp, _i, _i, _vp, _vp]),
    "pcv_mesh_backward": (_i, [_vp, _i, _i, _vp, _vp, _vp, _vp]),
    "pcv_dist_stats_workspace": (_i64, [_i]),
    "pcv_dist_stats": (_i, [_vp, _vp, _i64, _i, _i, _vp, _vp, _i64, _vp]),
    "pcv_kl_grad": (_i, [_vp, _vp, _vp, _i64, _i, _i, _vp, ctypes.c_double, _vp, _vp]),
    "pcv_prob_grad_to_amp": (_i, [_vp, _vp, _i64, _vp, _vp]),
    "pcv_distribution_static": (_i, [_vp, _i, _vp, _vp, _vp, _vp]),
    "pcv_distribution_static_max_bytes": (_i64, []),
    "pcv_amplitudes_multi": (_i, [_vp, _i, _i, _vp, _vp, _i64, _vp, _vp, _vp]),
    "pcv_gemm_bf16": (_i, [_vp, _i, _vp, _i, _i, _i, _i, _i, _vp, _vp, _i, _vp, _i, _vp, _i, _vp]),
    "pcv_gemm_bf16_tc": (_i, [_vp, _i, _vp, _i, _i, _i, _i, _i, _vp, _vp, _i, _vp, _i, _vp, _i, _vp, _vp]),
    "pcv_transpose_bf16": (_i, [_vp, _i, _i, _i, _vp, _i, _vp]),
    "pcv_colsum_bf16": (_i, [_vp, _i, _i, _i, _vp, _vp]),
    "pcv_phase_features": (_i, [_vp, _i, _i, _vp, _i, _vp]),
    "pcv_phase_features_grad": (_i, [_vp, _i, _i, _vp, _i, _vp, _vp]),
    "pcv_mse_workspace": (_i64, []),
    "pcv_mse": (_i, [_vp, _vp, _i64, _vp, _vp, _vp, _i64, _vp]),
    "pcv_adam": (_i, [_vp, _vp, _vp, _vp, _i64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _i,
                      _vp, _vp]),
    "pcv_f32_to_bf16": (_i, [_vp, _i64, _vp, _vp]),
    "pcv_log_f64_to_f32": (_i, [_vp, _i64, _vp, _vp]),
    "pcv_exp_f32_to_f64": (_i, [_vp, _i64, _vp, _vp]),
    "pcv_adam_f64": (_i, [_vp, _vp, _vp, _vp, _i64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                          ctypes.c_double, _i, _vp]),
    "pcv_amplitudes_backward_multi": (_i, [_vp, _i, _i, _vp, _vp, _i64, _vp, _vp, _vp, _i64, _vp]),
    "pcv_sample": (_i, [_vp, _i, _vp, _vp, _vp, _i64, _vp, _vp]),
    "pcv_fp64_probe": (_i, [_vp, _i, _i, _i, _vp]),
    "pcv_amplitudes_batched_workspace": (_i64, [_i, _i64]),
    "pcv_amplitudes_batched": (_i, [_vp, _i, _i64, _vp, _i64, _vp]),
    "pcv_amplitudes_batched_ex": (_i, [_vp, _i, _i64, _i, _vp, _i64, _vp]),
    "pcv_distribution_classes_workspace": (_i64, [_i, _i, _vp]),
    "pcv_distribution_classes": (_i, [_vp, _i, _i, _vp, _vp, _vp, _i64, _vp]),
    "pcv_distribution_source_size": (_i64, [_i, _i]),
    "pcv_distribution_source_workspace": (_i64, [_i, _vp]),
    "pcv_distribution_source": (_i, [_vp, _i, _vp, ctypes.c_double, ctypes.c_double, _vp, _vp, _i64, _vp]),
    "pcv_profile_enable": (_i, [_i]),
    "pcv_profile_read": (_i, [_vp, _vp, _i]),
    "pcv_launch_count": (_i64, []),
    "pcv_distribution_status": (_i, [_vp, _vp]),
    "pcv_set_wait_limit": (_i, [_i64]),
}

for _name, (_res, _args) in SIGNATURES.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class PcvError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.pcv_last_error().decode()
        super().__init__(f"{where} failed with code {code}: {msg}")
        self.code = code


def ptr(x):
    """Address of a torch tensor / numpy array / int / None for the C call."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _check(rc, where):
    if rc < 0:
        raise PcvError(int(rc), where)
    return rc


def _call(name, *args):
    return _check(getattr(_lib, name)(*args), name)


def pcv_version() -> str:
    return _lib.pcv_version().decode()


def pcv_last_error() -> str:
    return _lib.pcv_last_error().decode()


def pcv_num_outputs(m, n) -> int:
    return _call("pcv_num_outputs", m, n)


def pcv_unrank(m, n, idx, occ_out):
    return _call("pcv_unrank", m, n, idx, ptr(occ_out))


def pcv_rank(m, occ) -> int:
    return _call("pcv_rank", m, ptr(occ))


def pcv_amplitudes_workspace(m, n, n_out) -> int:
    return _call("pcv_amplitudes_workspace", m, n, n_out)


def pcv_amplitudes(U, m, input_occ, output_occ, n_out, amp, prob, workspace, workspace_bytes, stream):
    return _call("pcv_amplitudes", ptr(U), m, ptr(input_occ), ptr(output_occ), n_out, ptr(amp), ptr(prob),
                 ptr(workspace), workspace_bytes, stream)


def pcv_amplitudes_ex(U, m, input_occ, output_occ, n_out, amp, prob, algo, param, workspace, workspace_bytes, stream):
    return _call("pcv_amplitudes_ex", ptr(U), m, ptr(input_occ), ptr(output_occ), n_out, ptr(amp), ptr(prob),
                 algo, param, ptr(workspace), workspace_bytes, stream)


def pcv_amplitudes_ex_workspace(m, n, n_out, algo, param) -> int:
    return _call("pcv_amplitudes_ex_workspace", m, n, n_out, algo, param)


def pcv_distribution_workspace(m, n) -> int:
    return _call("pcv_distribution_workspace", m, n)


def pcv_distribution_tc_workspace(m, n) -> int:
    return _call("pcv_distribution_tc_workspace", m, n)


def pcv_distribution_auto_algo(m, n, workspace_bytes) -> int:
    return _call("pcv_distribution_auto_algo", m, n, workspace_bytes)


def pcv_distribution_workspace_min(m, n) -> int:
    return _call("pcv_distribution_workspace_min", m, n)


def pcv_distribution_range(U, m, input_occ, begin, end, prob, amp, workspace, workspace_bytes, stream):
    return _call("pcv_distribution_range", ptr(U), m, ptr(input_occ), begin, end, ptr(prob), ptr(amp),
                 ptr(workspace), workspace_bytes, stream)


def pcv_distribution_range_plan(m, n, begin, end):
    """[(pa[k], pb[k]) for k = 0..n]: the ranks of the low-side multisets whose
    outputs meet [begin, end)."""
    import numpy as np
    pa = np.zeros(n + 1, dtype=np.int64)
    pb = np.zeros(n + 1, dtype=np.int64)
    _call("pcv_distribution_range_plan", m, n, begin, end, pa.ctypes.data, pb.ctypes.data)
    return list(zip(pa.tolist(), pb.tolist()))


TC_BLOCK_FIELDS = ("kind", "rows_low", "tn", "rows0", "rows", "cols0", "cols", "row_off", "col_off", "lowoff",
                   "rs", "cs", "cge", "ri_off", "ci_off", "tile0")


def pcv_distribution_tc_blocks(m, n, begin=0, end=-1):
    """(header dict, [block dicts]): the output blocks of the tensor-core
    products for the outputs [begin, end) (host only; layout in include/pcv.h)."""
    import numpy as np
    need = ctypes.c_int64(0)
    _call("pcv_distribution_tc_blocks", m, n, begin, end, None, 0, ctypes.addressof(need))
    out = np.zeros(need.value, dtype=np.int64)
    _call("pcv_distribution_tc_blocks", m, n, begin, end, out.ctypes.data, out.size, None)
    h = out[:48].tolist()
    head = {"e": h[0], "L": h[1], "h": h[2], "blocks": h[3], "tiles": h[4], "ncols": h[5],
            "rows_off": h[6:8], "nrows": h[8:10], "cols_off": h[10:12], "wdig": h[12:14],
            "lev": [h[16:32], h[32:48]]}
    blocks = [dict(zip(TC_BLOCK_FIELDS, out[48 + 16 * b: 64 + 16 * b].tolist())) for b in range(h[3])]
    return head, blocks


def pcv_distribution(U, m, input_occ, prob, amp, workspace, workspace_bytes, stream):
    return _call("pcv_distribution", ptr(U), m, ptr(input_occ), ptr(prob), ptr(amp), ptr(workspace),
                 workspace_bytes, stream)


def pcv_distribution_ex(U, m, input_occ, prob, amp, algo, param, workspace, workspace_bytes, stream):
    return _call("pcv_distribution_ex", ptr(U), m, ptr(input_occ), ptr(prob), ptr(amp), algo, param,
                 ptr(workspace), workspace_bytes, stream)


class pcv_batch_desc(ctypes.Structure):
    """Mirror of the C struct pcv_batch_desc (include/pcv.h)."""
    _fields_ = [("U", _vp), ("outputs", _vp), ("amp", _vp), ("prob", _vp), ("n_out", _i64),
                ("m", ctypes.c_int32), ("n", ctypes.c_int32), ("cols", ctypes.c_int32 * PCV_MAX_PHOTONS)]


def pcv_amplitudes_batched_workspace(n_circ, total_outputs) -> int:
    return _call("pcv_amplitudes_batched_workspace", n_circ, total_outputs)


def pcv_amplitudes_batched(descs, n_circ, total_outputs, workspace, workspace_bytes, stream):
    return _call("pcv_amplitudes_batched", ptr(descs), n_circ, total_outputs, ptr(workspace), workspace_bytes, stream)


def pcv_amplitudes_batched_ex(descs, n_circ, total_outputs, algo, workspace, workspace_bytes, stream):
    return _call("pcv_amplitudes_batched_ex", ptr(descs), n_circ, total_outputs, algo, ptr(workspace),
                 workspace_bytes, stream)


def pcv_distribution_classes_workspace(m, G, class_occ) -> int:
    return _call("pcv_distribution_classes_workspace", m, G, ptr(class_occ))


def pcv_distribution_classes(U, m, G, class_occ, prob, workspace, workspace_bytes, stream):
    return _call("pcv_distribution_classes", ptr(U), m, G, ptr(class_occ), ptr(prob), ptr(workspace),
                 workspace_bytes, stream)


def pcv_distribution_source_size(m, n) -> int:
    return _call("pcv_distribution_source_size", m, n)


def pcv_distribution_source_workspace(m, input_occ) -> int:
    return _call("pcv_distribution_source_workspace", m, ptr(input_occ))


def pcv_distribution_source(U, m, input_occ, transmittance, indistinguishability, prob, workspace,
                            workspace_bytes, stream):
    return _call("pcv_distribution_source", ptr(U), m, ptr(input_occ), float(transmittance),
                 float(indistinguishability), ptr(prob), ptr(workspace), workspace_bytes, stream)


def pcv_distribution_batched_workspace(B, m, n) -> int:
    return _call("pcv_distribution_batched_workspace", B, m, n)


def pcv_distribution_batched(U, B, m, input_occ, prob, amp, workspace, workspace_bytes, stream):
    return _call("pcv_distribution_batched", ptr(U), B, m, ptr(input_occ), ptr(prob), ptr(amp), ptr(workspace),
                 workspace_bytes, stream)


def pcv_amplitudes_backward_workspace(B, m, n, n_out) -> int:
    return _call("pcv_amplitudes_backward_workspace", B, m, n, n_out)


def pcv_amplitudes_backward(U, m, input_occ, output_occ, n_out, grad_amp, grad_U, workspace, workspace_bytes,
                            stream):
    return _call("pcv_amplitudes_backward", ptr(U), m, ptr(input_occ), ptr(output_occ), n_out, ptr(grad_amp),
                 ptr(grad_U), ptr(workspace), workspace_bytes, stream)


def pcv_distribution_backward_workspace(B, m, n) -> int:
    return _call("pcv_distribution_backward_workspace", B, m, n)


def pcv_distribution_backward(U, B, m, input_occ, grad_amp, grad_U, workspace, workspace_bytes, stream):
    return _call("pcv_distribution_backward", ptr(U), B, m, ptr(input_occ), ptr(grad_amp), ptr(grad_U),
                 ptr(workspace), workspace_bytes, stream)


def pcv_mesh_unitary(phases, B, m, U, stream):
    return _call("pcv_mesh_unitary", ptr(phases), B, m, ptr(U), stream)


def pcv_mesh_backward(phases, B, m, U, grad_U, grad_phases, stream):
    return _call("pcv_mesh_backward", ptr(phases), B, m, ptr(U), ptr(grad_U), ptr(grad_phases), stream)


def pcv_dist_stats_workspace(B) -> int:
    return _call("pcv_dist_stats_workspace", B)


def pcv_dist_stats(p, q, N, B, q_batched, out, workspace, workspace_bytes, stream):
    return _call("pcv_dist_stats", ptr(p), ptr(q), N, B, q_batched, ptr(out), ptr(workspace), workspace_bytes, stream)


def pcv_kl_grad(p, q, amp, N, B, q_batched, batch_scale, scale, grad_amp, stream):
    return _call("pcv_kl_grad", ptr(p), ptr(q), ptr(amp), N, B, q_batched, ptr(batch_scale), scale, ptr(grad_amp),
                 stream)


def pcv_prob_grad_to_amp(grad_prob, amp, count, grad_amp, stream):
    return _call("pcv_prob_grad_to_amp", ptr(grad_prob), ptr(amp), count, ptr(grad_amp), stream)


def pcv_distribution_static(U, m, input_occ, prob, amp, stream):
    return _call("pcv_distribution_static", ptr(U), m, ptr(input_occ), ptr(prob), ptr(amp), stream)


def pcv_distribution_static_max_bytes() -> int:
    return _call("pcv_distribution_static_max_bytes")


def pcv_amplitudes_multi(U, B, m, input_occ, output_occ, n_out, amp, prob, stream):
    return _call("pcv_amplitudes_multi", ptr(U), B, m, ptr(input_occ), ptr(output_occ), n_out, ptr(amp), ptr(prob),
                 stream)


def pcv_gemm_bf16(A, lda, B, ldb, M, N, K, mode, bias, outf, ldo, outb, ldob, pre, ldp, stream):
    return _call("pcv_gemm_bf16", ptr(A), lda, ptr(B), ldb, M, N, K, mode, ptr(bias), ptr(outf), ldo, ptr(outb),
                 ldob, ptr(pre), ldp, stream)


def pcv_gemm_bf16_tc(A, lda, B, ldb, M, N, K, mode, bias, outf, ldo, outb, ldob, pre, ldp, error, stream):
    return _call("pcv_gemm_bf16_tc", ptr(A), lda, ptr(B), ldb, M, N, K, mode, ptr(bias), ptr(outf), ldo, ptr(outb),
                 ldob, ptr(pre), ldp, ptr(error), stream)


def pcv_transpose_bf16(inp, R, C, ldi, out, ldo, stream):
    return _call("pcv_transpose_bf16", ptr(inp), R, C, ldi, ptr(out), ldo, stream)


def pcv_colsum_bf16(dY, M, N, ld, db, stream):
    return _call("pcv_colsum_bf16", ptr(dY), M, N, ld, ptr(db), stream)


def pcv_phase_features(phases, B, P, X, ldx, stream):
    return _call("pcv_phase_features", ptr(phases), B, P, ptr(X), ldx, stream)


def pcv_phase_features_grad(phases, B, P, dX, ldx, grad_phases, stream):
    return _call("pcv_phase_features_grad", ptr(phases), B, P, ptr(dX), ldx, ptr(grad_phases), stream)


def pcv_mse_workspace() -> int:
    return _call("pcv_mse_workspace")


def pcv_mse(pred, target, count, loss, grad_pred_bf16, workspace, workspace_bytes, stream):
    return _call("pcv_mse", ptr(pred), ptr(target), count, ptr(loss), ptr(grad_pred_bf16), ptr(workspace),
                 workspace_bytes, stream)


def pcv_adam(w, m, v, g, count, lr, beta1, beta2, eps, step, w_bf16, stream):
    return _call("pcv_adam", ptr(w), ptr(m), ptr(v), ptr(g), count, lr, beta1, beta2, eps, step, ptr(w_bf16), stream)


def pcv_f32_to_bf16(inp, count, out, stream):
    return _call("pcv_f32_to_bf16", ptr(inp), count, ptr(out), stream)


def pcv_log_f64_to_f32(inp, count, out, stream):
    return _call("pcv_log_f64_to_f32", ptr(inp), count, ptr(out), stream)


def pcv_exp_f32_to_f64(inp, count, out, stream):
    return _call("pcv_exp_f32_to_f64", ptr(inp), count, ptr(out), stream)


def pcv_adam_f64(w, m, v, g, count, lr, beta1, beta2, eps, step, stream):
    return _call("pcv_adam_f64", ptr(w), ptr(m), ptr(v), ptr(g), count, lr, beta1, beta2, eps, step, stream)


def pcv_amplitudes_backward_multi(U, B, m, input_occ, output_occ, n_out, grad_amp, grad_U, workspace,
                                  workspace_bytes, stream):
    return _call("pcv_amplitudes_backward_multi", ptr(U), B, m, ptr(input_occ), ptr(output_occ), n_out,
                 ptr(grad_amp), ptr(grad_U), ptr(workspace), workspace_bytes, stream)


def pcv_distribution_slos_workspace(B, m, n) -> int:
    return _call("pcv_distribution_slos_workspace", B, m, n)


def pcv_distribution_slos(U, B, m, input_occ, prob, amp, workspace, workspace_bytes, stream):
    return _call("pcv_distribution_slos", ptr(U), B, m, ptr(input_occ), ptr(prob), ptr(amp), ptr(workspace),
                 workspace_bytes, stream)


def pcv_sample(U, m, input_occ, perm, uniforms, count, samples, stream):
    return _call("pcv_sample", ptr(U), m, ptr(input_occ), ptr(perm), ptr(uniforms), count, ptr(samples), stream)


def pcv_fp64_probe(out, blocks, threads, iters, stream):
    return _call("pcv_fp64_probe", ptr(out), blocks, threads, iters, stream)


STAGES = ("dist_tables", "dist_products", "glynn_plain", "tc_split", "tc_edge_fp64")


def pcv_profile_enable(on: bool):
    return _call("pcv_profile_enable", 1 if on else 0)


def pcv_profile_read():
    """{stage name: (milliseconds, calls)} accumulated since the last read."""
    import numpy as np
    ms = np.zeros(len(STAGES))
    calls = np.zeros(len(STAGES), dtype=np.int64)
    _call("pcv_profile_read", ms.ctypes.data, calls.ctypes.data, len(STAGES))
    return {k: (float(ms[i]), int(calls[i])) for i, k in enumerate(STAGES)}


def pcv_launch_count() -> int:
    return int(_lib.pcv_launch_count())


def pcv_distribution_status(workspace, stream):
    return _call("pcv_distribution_status", ptr(workspace), stream)


def pcv_set_wait_limit(polls):
    return _call("pcv_set_wait_limit", polls)
