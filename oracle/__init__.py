"""CPU FP64 oracle for the amplitude path (Sec. 4.2, Eq. eqperm) and its companions.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline / reference leg are the only callers.  Nothing here is
shared with, or called by, the CUDA library; the only common module is the
seeded input generator ``pcv_inputs``.

Contents
--------
* ``perm_leibniz``, ``perm_ryser``, ``perm_ryser_dd``: the permanent by its
  definition, by Ryser's formula, and by Ryser's formula in double-double
  arithmetic (plain C, ``pcv_oracle.c``).
* ``amplitude``, ``amplitudes``, ``distribution``: Eq. eqperm over explicit
  outputs or the whole output space S_{m,n} in canonical order.
* ``enumerate_outputs``, ``num_outputs``: canonical order = lexicographic
  order of the non-decreasing photon->mode list.
* ``amplitude_grad``: dA/dU by the Laplace expansion (minor permanents).
* ``mesh``: Clements-layout MZI mesh unitary U(phi) (Sec. 2, Eq. bs, MZI of
  Sec. 4.2's listing), numpy.
* ``tvd``, ``kl``: Eq. bosonsampling's total variation distance; KL(q||p).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain IEEE double, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            u8 = ctypes.POINTER(ctypes.c_uint8)
            lib.oracle_perm_leibniz.argtypes = [ctypes.c_int, dp, dp]
            lib.oracle_perm_ryser.argtypes = [ctypes.c_int, dp, dp]
            lib.oracle_perm_ryser_dd.argtypes = [ctypes.c_int, dp, dp]
            lib.oracle_amplitude.argtypes = [ctypes.c_int, dp, u8, u8, ctypes.c_int, dp]
            lib.oracle_amplitudes.argtypes = [ctypes.c_int, dp, u8, u8, ctypes.c_int64, ctypes.c_int, dp]
            lib.oracle_num_outputs.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.oracle_num_outputs.restype = ctypes.c_int64
            lib.oracle_enumerate.argtypes = [ctypes.c_int, ctypes.c_int, u8, ctypes.c_int64]
            lib.oracle_enumerate.restype = ctypes.c_int64
            lib.oracle_distribution.argtypes = [ctypes.c_int, dp, u8, dp, dp]
            lib.oracle_distribution.restype = ctypes.c_int
            lib.oracle_amplitude_grad.argtypes = [ctypes.c_int, dp, u8, u8, dp]
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _cmat(A):
    return np.ascontiguousarray(A, dtype=np.complex128)


def num_threads() -> int:
    return int(_L().oracle_num_threads())


def perm_leibniz(A) -> complex:
    """Permanent by definition: sum over permutations of prod_i A[i, sigma(i)]."""
    A = _cmat(A)
    n = A.shape[0]
    assert A.shape == (n, n) and n <= 12
    out = np.zeros(2)
    _L().oracle_perm_leibniz(n, _dp(A), _dp(out))
    return complex(out[0], out[1])


def perm_ryser(A) -> complex:
    """Permanent by Ryser's formula (Sec. 3.2.3)."""
    A = _cmat(A)
    n = A.shape[0]
    assert A.shape == (n, n) and n <= 40
    out = np.zeros(2)
    _L().oracle_perm_ryser(n, _dp(A), _dp(out))
    return complex(out[0], out[1])


def perm_ryser_dd(A) -> complex:
    """Ryser's formula evaluated in double-double arithmetic (about 106 bits),
    for sizes where the plain double sum loses digits to cancellation."""
    A = _cmat(A)
    n = A.shape[0]
    assert A.shape == (n, n) and n <= 40
    out = np.zeros(2)
    _L().oracle_perm_ryser_dd(n, _dp(A), _dp(out))
    return complex(out[0], out[1])


_METHODS = {"ryser": 0, "leibniz": 1, "ryser_dd": 2}


def amplitude(U, input_occ, output_occ, method: str = "ryser") -> complex:
    """a(S) = Perm(U_{T,S}) / sqrt(prod s! prod t!) (Eq. eqperm)."""
    U = _cmat(U)
    m = U.shape[0]
    t = np.ascontiguousarray(input_occ, dtype=np.uint8)
    s = np.ascontiguousarray(output_occ, dtype=np.uint8)
    out = np.zeros(2)
    _L().oracle_amplitude(m, _dp(U), _u8(t), _u8(s), _METHODS[method], _dp(out))
    return complex(out[0], out[1])


def amplitudes(U, input_occ, outputs, method: str = "ryser") -> np.ndarray:
    """Eq. eqperm for each row of ``outputs`` (uint8 [n_out, m]); complex128 [n_out]."""
    U = _cmat(U)
    m = U.shape[0]
    t = np.ascontiguousarray(input_occ, dtype=np.uint8)
    s = np.ascontiguousarray(outputs, dtype=np.uint8).reshape(-1, m)
    amp = np.zeros(s.shape[0], dtype=np.complex128)
    _L().oracle_amplitudes(m, _dp(U), _u8(t), _u8(s), s.shape[0],
                           _METHODS[method], _dp(amp.view(np.float64)))
    return amp


def num_outputs(m: int, n: int) -> int:
    """|S_{m,n}| = C(m+n-1, n)."""
    return int(_L().oracle_num_outputs(m, n))


def enumerate_outputs(m: int, n: int) -> np.ndarray:
    """uint8 [C(m+n-1,n), m], canonical (lexicographic non-decreasing mode list) order."""
    N = num_outputs(m, n)
    occ = np.zeros((N, m), dtype=np.uint8)
    got = _L().oracle_enumerate(m, n, _u8(occ), N)
    assert got == N
    return occ


def enumerate_outputs_prefix(m: int, n: int, count: int) -> np.ndarray:
    """The first min(count, C(m+n-1,n)) outputs of the canonical order."""
    N = min(count, num_outputs(m, n))
    occ = np.zeros((N, m), dtype=np.uint8)
    _L().oracle_enumerate(m, n, _u8(occ), N)
    return occ


def distribution(U, input_occ):
    """(prob float64[N], amp complex128[N]) over all outputs in canonical order."""
    U = _cmat(U)
    m = U.shape[0]
    t = np.ascontiguousarray(input_occ, dtype=np.uint8)
    N = num_outputs(m, int(t.sum()))
    prob = np.zeros(N)
    amp = np.zeros(N, dtype=np.complex128)
    rc = _L().oracle_distribution(m, _dp(U), _u8(t), _dp(prob), _dp(amp.view(np.float64)))
    assert rc == 0
    return prob, amp


def amplitude_grad(U, input_occ, output_occ) -> np.ndarray:
    """D[k, l] = d a(S) / d U[k, l] (holomorphic derivative), complex128 [m, m]."""
    U = _cmat(U)
    m = U.shape[0]
    t = np.ascontiguousarray(input_occ, dtype=np.uint8)
    s = np.ascontiguousarray(output_occ, dtype=np.uint8)
    D = np.zeros((m, m), dtype=np.complex128)
    _L().oracle_amplitude_grad(m, _dp(U), _u8(t), _u8(s), _dp(D.view(np.float64)))
    return D


def grad_U_from_amp_grad(U, input_occ, outputs, grad_amp) -> np.ndarray:
    """grad_U = sum_s gbar_s * conj(d a_s / dU), the gradient of a real loss in
    the dL/dRe + i dL/dIm convention, given gbar_s for each output amplitude."""
    G = np.zeros((U.shape[0], U.shape[0]), dtype=np.complex128)
    for s, g in zip(np.asarray(outputs), np.asarray(grad_amp)):
        if g != 0:
            G += g * np.conj(amplitude_grad(U, input_occ, s))
    return G


# ----------------------------------------------------------------- mesh

#: balanced beam splitter in the Rx convention at theta = pi/2 (Eq. bs)
BS_RX_HALF = np.array([[1.0, 1.0j], [1.0j, 1.0]], dtype=np.complex128) / np.sqrt(2.0)


def mzi(phi_a: float, phi_b: float) -> np.ndarray:
    """2x2 unitary of BS, then PS(phi_a) on the first mode, then BS, then
    PS(phi_b) on the second mode (the MZI of Sec. 4.2's Boson-sampling code);
    later components multiply on the left."""
    ps_a = np.diag([np.exp(1j * phi_a), 1.0])
    ps_b = np.diag([1.0, np.exp(1j * phi_b)])
    return ps_b @ BS_RX_HALF @ ps_a @ BS_RX_HALF


def clements_pairs(m: int):
    """MZI positions of the rectangular (Clements) mesh: m columns; column c
    holds MZIs on modes (k, k+1) for k = c mod 2, c mod 2 + 2, ... < m-1."""
    pairs = []
    for c in range(m):
        for k in range(c % 2, m - 1, 2):
            pairs.append(k)
    return pairs


def mesh(phases) -> np.ndarray:
    """U(phi) of the Clements mesh; phases[2*q], phases[2*q+1] = (phi_a, phi_b) of MZI q."""
    phases = np.asarray(phases, dtype=np.float64)
    n_mzi = phases.shape[0] // 2
    m = 2
    while len(clements_pairs(m)) < n_mzi:
        m += 1
    assert len(clements_pairs(m)) == n_mzi, "phase count is not a Clements mesh"
    U = np.eye(m, dtype=np.complex128)
    for q, k in enumerate(clements_pairs(m)):
        T = np.eye(m, dtype=np.complex128)
        T[k:k + 2, k:k + 2] = mzi(phases[2 * q], phases[2 * q + 1])
        U = T @ U
    return U


# ------------------------------------------------------- distributions

def tvd(p, q) -> float:
    """Total variation distance (Eq. bosonsampling): 1/2 sum |p - q|."""
    return 0.5 * float(np.sum(np.abs(np.asarray(p, np.float64) - np.asarray(q, np.float64))))


def kl(q, p) -> float:
    """KL(q || p) = sum q log(q / p) over q > 0."""
    q = np.asarray(q, np.float64)
    p = np.asarray(p, np.float64)
    nz = q > 0
    return float(np.sum(q[nz] * (np.log(q[nz]) - np.log(p[nz]))))
