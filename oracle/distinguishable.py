"""CPU FP64 oracle for partially distinguishable photons.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): the tests,
``__graft_entry__.smoke()`` and the bench's CPU legs are the only callers; the
CUDA library shares nothing with this file.

The paper's Processor takes a source with a transmittance and an
indistinguishability (Sec. processors, "Processors"), and its Hong-Ou-Mandel
experiment (Sec. hom) simulates such a source, but the paper prints no
formula for either. The models below are written from the physics.

Photon classes.  The input photons are split into classes. Photons of one
class are identical. Photons of different classes are perfectly
distinguishable: they have orthogonal internal states, and the detectors only
count photons per mode. Each class then evolves on its own. With
P_g(S_g) = |Perm(U_{S_g,T_g})|^2 / (prod s_g! prod t_g!) (Eq. eqperm for
class g alone),

    P(S) = sum over S_1 + ... + S_G = S, |S_g| = n_g, of prod_g P_g(S_g).

``class_distribution`` evaluates exactly this sum. It combines the classes
one at a time: every pair of outcomes of the classes so far and of the next
class is added to the bin of their summed occupation.

Source indistinguishability.  Each photon is independently "pure" with
probability q and otherwise "noisy". The pure photons form one class. Every
noisy photon is a class of its own. So

    P(S) = sum over subsets D of the photons of q^{n-|D|} (1-q)^{|D|} P_{classes(D)}(S).

Two photons on a 50:50 beam splitter then coincide with probability
(1 - q^2)/2, a HOM visibility of q^2. A source of indistinguishability
(visibility) V therefore takes q = sqrt(V).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import distribution, enumerate_outputs, perm_ryser


def _index(m: int, n: int):
    """Map from an occupation (bytes) to its canonical index in S_{m,n}."""
    occ = enumerate_outputs(m, n)
    return {occ[i].tobytes(): i for i in range(occ.shape[0])}, occ


def class_distribution(U, classes) -> np.ndarray:
    """P(S) over S_{m,n} in canonical order for photon classes.

    classes: sequence of uint8[m] input occupations, one per class (a class
    may be empty); n = total photon number."""
    U = np.asarray(U, dtype=np.complex128)
    m = U.shape[0]
    classes = [np.asarray(t, dtype=np.uint8) for t in classes]
    cur_n = 0
    cur_p = np.ones(1)
    cur_occ = np.zeros((1, m), dtype=np.int64)
    for t in classes:
        k = int(t.sum())
        if k == 0:
            continue
        p_g, _ = distribution(U, t)
        occ_g = enumerate_outputs(m, k).astype(np.int64)
        idx, occ_new = _index(m, cur_n + k)
        new_p = np.zeros(occ_new.shape[0])
        for a in range(cur_p.shape[0]):
            if cur_p[a] == 0.0:
                continue
            summed = occ_g + cur_occ[a][None, :]
            for b in range(occ_g.shape[0]):
                new_p[idx[summed[b].astype(np.uint8).tobytes()]] += cur_p[a] * p_g[b]
        cur_n += k
        cur_p, cur_occ = new_p, occ_new.astype(np.int64)
    return cur_p


def distinguishable_closed_form(U, input_occ, output_occ) -> float:
    """All photons mutually distinguishable: P(S) = Perm(W_{S,T}) / prod s!,
    with W = |U|^2 elementwise, rows repeated by S and one column per photon."""
    U = np.asarray(U, dtype=np.complex128)
    W = np.abs(U) ** 2
    rows = np.repeat(np.arange(U.shape[0]), np.asarray(output_occ, dtype=np.int64))
    cols = np.repeat(np.arange(U.shape[0]), np.asarray(input_occ, dtype=np.int64))
    if len(rows) != len(cols):
        return 0.0
    sub = W[np.ix_(rows, cols)].astype(np.complex128)
    fs = math.prod(math.factorial(int(s)) for s in output_occ)
    return float(perm_ryser(sub).real) / fs


def photon_modes(input_occ) -> list[int]:
    """Input mode of each photon (the sorted photon -> mode list)."""
    return [int(c) for c in np.repeat(np.arange(len(input_occ)), np.asarray(input_occ, dtype=np.int64))]


def classes_for_noisy(input_occ, noisy) -> list[np.ndarray]:
    """Classes when the photons listed in `noisy` (indices into photon_modes)
    are distinguishable from everything: the pure ones first, then one class
    per noisy photon."""
    m = len(input_occ)
    modes = photon_modes(input_occ)
    pure = np.zeros(m, dtype=np.uint8)
    out = []
    for k, c in enumerate(modes):
        if k in noisy:
            t = np.zeros(m, dtype=np.uint8)
            t[c] = 1
            out.append(t)
        else:
            pure[c] += 1
    return [pure] + out


def source_distribution(U, input_occ, q: float) -> np.ndarray:
    """P(S) over S_{m,n} when each photon is pure with probability q (see the
    module docstring): the mixture over every subset of noisy photons."""
    n = int(np.asarray(input_occ).sum())
    total = None
    for size in range(n + 1):
        for noisy in itertools.combinations(range(n), size):
            w = q ** (n - size) * (1.0 - q) ** size
            if w == 0.0:
                continue
            p = w * class_distribution(U, classes_for_noisy(input_occ, set(noisy)))
            total = p if total is None else total + p
    return total


def lossy_source_distribution(U, input_occ, eta: float, q: float) -> np.ndarray:
    """Photon-number-resolved distribution of a lossy, partially
    distinguishable source: each photon independently is absent (probability
    1 - eta), pure (eta q) or noisy (eta (1 - q)).  The pure photons form one
    class, every noisy photon a class of its own (module docstring).

    Returns P over S_{m,0}, S_{m,1}, ..., S_{m,n} concatenated in that order,
    each block in canonical order; the blocks sum to 1 together."""
    U = np.asarray(U, dtype=np.complex128)
    m = U.shape[0]
    modes = photon_modes(input_occ)
    n = len(modes)
    blocks = [np.zeros(math.comb(m + k - 1, k)) for k in range(n + 1)]
    for state in itertools.product(range(3), repeat=n):       # 0 absent, 1 pure, 2 noisy
        w = 1.0
        for st in state:
            w *= (1.0 - eta) if st == 0 else (eta * q if st == 1 else eta * (1.0 - q))
        if w == 0.0:
            continue
        pure = np.zeros(m, dtype=np.uint8)
        classes = []
        for k, st in enumerate(state):
            if st == 1:
                pure[modes[k]] += 1
            elif st == 2:
                e = np.zeros(m, dtype=np.uint8)
                e[modes[k]] = 1
                classes.append(e)
        kept = sum(1 for st in state if st != 0)
        blocks[kept] += w * class_distribution(U, [pure] + classes)
    return np.concatenate(blocks)
