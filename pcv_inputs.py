"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module draws random numbers and lays them out; it holds none of the
amplitude arithmetic (no permanent, no normalisation, no enumeration of the
output space).  Both the CPU oracle and the CUDA path receive exactly the
arrays produced here.

Workload recipe (the paper's Boson-sampling workload, Sec. 4.2: Haar-random
m x m unitaries, single photons in distinct input modes):

* Haar unitary: QR decomposition of an m x m matrix of i.i.d. complex
  Gaussians N(0,1/2) + i N(0,1/2), with the phases of R's diagonal moved into
  Q (Sec. 4.2 cites a Haar recipe without fixing one; this is the standard
  Mezzadri construction).
* Input state: one photon in each of modes 0..n-1 unless stated otherwise.
* Explicit output sets: n <= 16 draws a uniform n-subset of the m modes
  (collision-free); n > 16 draws a uniform multiset by stars and bars (a
  uniform n-subset of m+n-1 slots).
* Mesh phases: i.i.d. uniform on [0, 2*pi).
* KL targets: Dirichlet(1) over the output set.
"""
from __future__ import annotations

import numpy as np

#: base seed of the named workloads; workload k uses BASE_SEED + k
BASE_SEED = 2204006020


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


def haar_unitary(m: int, seed: int) -> np.ndarray:
    """Haar-random m x m complex128 unitary, row = output mode, column = input mode."""
    g = rng(seed)
    z = (g.standard_normal((m, m)) + 1j * g.standard_normal((m, m))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    ph = d / np.abs(d)
    return np.ascontiguousarray(q * ph[None, :], dtype=np.complex128)


def random_complex_matrix(rows: int, cols: int, seed: int) -> np.ndarray:
    """i.i.d. complex Gaussian matrix (not unitary) for permanent identities."""
    g = rng(seed)
    z = (g.standard_normal((rows, cols)) + 1j * g.standard_normal((rows, cols))) / np.sqrt(2.0)
    return np.ascontiguousarray(z, dtype=np.complex128)


def single_photon_input(m: int, n: int, modes=None) -> np.ndarray:
    """Occupation vector uint8[m] with one photon in each listed mode (default 0..n-1)."""
    occ = np.zeros(m, dtype=np.uint8)
    for k in (range(n) if modes is None else modes):
        occ[k] += 1
    return occ


def random_outputs(m: int, n: int, count: int, seed: int) -> np.ndarray:
    """uint8[count, m] occupation vectors with n photons each.

    n <= 16: a uniform random n-subset of modes (no collisions).
    n > 16: a uniform random multiset via stars and bars.  Duplicates among
    the `count` rows are allowed.
    """
    g = rng(seed)
    out = np.zeros((count, m), dtype=np.uint8)
    if count == 0 or n == 0:
        return out
    rows = np.repeat(np.arange(count), n)
    if n <= 16 and n <= m:
        modes = np.argsort(g.random((count, m)), axis=1)[:, :n]          # uniform n-subsets
        out[rows, modes.reshape(-1)] = 1
    else:
        slots = np.sort(np.argsort(g.random((count, m + n - 1)), axis=1)[:, :n], axis=1)
        modes = slots - np.arange(n)[None, :]                               # stars and bars
        np.add.at(out, (rows, modes.reshape(-1)), 1)
    return out


def random_bunched_outputs(m: int, n: int, count: int, seed: int) -> np.ndarray:
    """uint8[count, m]: uniform random multisets (bunched outputs allowed) for any n."""
    g = rng(seed)
    out = np.zeros((count, m), dtype=np.uint8)
    if count == 0 or n == 0:
        return out
    slots = np.sort(np.argsort(g.random((count, m + n - 1)), axis=1)[:, :n], axis=1)
    np.add.at(out, (np.repeat(np.arange(count), n), (slots - np.arange(n)[None, :]).reshape(-1)), 1)
    return out


def mesh_phases(batch: int, n_phases: int, seed: int) -> np.ndarray:
    """float64[batch, n_phases] uniform on [0, 2*pi)."""
    return rng(seed).uniform(0.0, 2.0 * np.pi, size=(batch, n_phases))


def dirichlet_target(size: int, seed: int) -> np.ndarray:
    """float64[size] Dirichlet(1) probability vector."""
    return rng(seed).dirichlet(np.ones(size))


def batched_circuits(n_circ: int, m_lo: int, m_hi: int, n_lo: int, n_hi: int,
                     outputs_per_circ: int, seed: int):
    """Uneven batch: per circuit m ~ U{m_lo..m_hi}, n ~ U{n_lo..min(n_hi, m)},
    Haar U (seed + 1000 + c), photons in modes 0..n-1, random outputs (seed + 5000 + c).

    Returns a list of dicts {m, n, U, input_occ, outputs}.
    """
    g = rng(seed)
    circs = []
    for c in range(n_circ):
        m = int(g.integers(m_lo, m_hi + 1))
        n = int(g.integers(n_lo, min(n_hi, m) + 1))
        circs.append(dict(
            m=m, n=n,
            U=haar_unitary(m, seed + 1000 + c),
            input_occ=single_photon_input(m, n),
            outputs=random_outputs(m, n, outputs_per_circ, seed + 5000 + c),
        ))
    return circs


def sampler_randomness(count: int, n: int, seed: int):
    """(perm uint8[count, n], uniforms float64[count, n]): a uniform random
    permutation of the n photons and one uniform number per photon per sample."""
    g = rng(seed)
    perm = np.argsort(g.random((count, n)), axis=1).astype(np.uint8)
    return perm, g.random((count, n))
