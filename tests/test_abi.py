"""CPU checks of the C-ABI library: it builds, loads, exports every symbol
include/pcv.h declares, and its host-only helpers (output-space counting,
ranking, argument validation) behave.  No compute call reaches the GPU."""
import ctypes
import itertools
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_build_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "pcv_build", os.path.join(ROOT, "paper_2204_00602_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module", autouse=True)
def lib():
    path = load_build_module().build()
    return ctypes.CDLL(path)


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(pcv_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for want in ("pcv_amplitudes", "pcv_distribution", "pcv_num_outputs", "pcv_unrank", "pcv_last_error"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol(lib):
    from paper_2204_00602_gb300 import _abi
    assert set(declared_functions()) <= set(_abi.SIGNATURES)


def test_num_outputs_and_errors(lib):
    from paper_2204_00602_gb300 import _abi
    assert _abi.pcv_num_outputs(20, 10) == 20_030_010
    assert _abi.pcv_num_outputs(6, 3) == 56
    assert _abi.pcv_num_outputs(1, 30) == 1
    assert _abi.pcv_num_outputs(5, 0) == 1
    with pytest.raises(_abi.PcvError) as e:
        _abi.pcv_num_outputs(0, 3)
    assert e.value.code == _abi.PCV_EINVAL
    with pytest.raises(_abi.PcvError) as e:
        _abi.pcv_num_outputs(1024, 30)
    assert e.value.code == _abi.PCV_ERANGE


@pytest.mark.parametrize("m,n", [(6, 3), (4, 2), (5, 5), (7, 1), (3, 0)])
def test_unrank_and_rank_follow_lexicographic_order(m, n):
    import oracle
    import paper_2204_00602_gb300 as pcv
    occ = oracle.enumerate_outputs(m, n)
    for i, o in enumerate(occ):
        assert np.array_equal(pcv.unrank(m, n, i), o)
        assert pcv.rank(o) == i


def test_rank_of_a_large_space_round_trips():
    import paper_2204_00602_gb300 as pcv
    m, n = 20, 10
    N = pcv.num_outputs(m, n)
    for idx in (0, 1, 12345, N // 2, N - 2, N - 1):
        assert pcv.rank(pcv.unrank(m, n, idx)) == idx
    assert list(np.nonzero(pcv.unrank(m, n, N - 1))[0]) == [m - 1]
    first = pcv.unrank(m, n, 0)
    assert first[0] == n


def test_unrank_out_of_range():
    from paper_2204_00602_gb300 import _abi
    occ = np.zeros(6, np.uint8)
    with pytest.raises(_abi.PcvError) as e:
        _abi.pcv_unrank(6, 3, 56, occ)
    assert e.value.code == _abi.PCV_ERANGE


def test_argument_errors_are_reported_before_any_launch():
    from paper_2204_00602_gb300 import _abi
    t = np.array([1, 1, 0], np.uint8)
    fake = 1 << 40        # never dereferenced: validation fails first
    cases = [
        (dict(U=None, m=3), _abi.PCV_EINVAL),
        (dict(U=fake, m=0), _abi.PCV_EINVAL),
        (dict(U=fake + 8, m=3), _abi.PCV_EINVAL),          # misaligned U
        (dict(U=fake, m=3, n_out=-1), _abi.PCV_EINVAL),
        (dict(U=fake, m=3, amp=None, prob=None), _abi.PCV_EINVAL),
        (dict(U=fake, m=3, algo=_abi.PCV_ALGO_GROUP, param=3), _abi.PCV_EINVAL),
        (dict(U=fake, m=3, algo=_abi.PCV_ALGO_GROUP, param=4), _abi.PCV_EINVAL),   # 4 > 2^(n-1)
        (dict(U=fake, m=3, algo=_abi.PCV_ALGO_BLOCK, param=1), _abi.PCV_EINVAL),   # n < 9
        (dict(U=fake, m=3, algo=_abi.PCV_ALGO_MULT, param=-1), _abi.PCV_EINVAL),
        (dict(U=fake, m=3, algo=_abi.PCV_ALGO_MULT, param=1025), _abi.PCV_EINVAL),
        (dict(U=fake, m=3, algo=_abi.PCV_ALGO_MULT, param=4), _abi.PCV_ENOMEM),    # partial sums need workspace
    ]
    for kw, code in cases:
        a = dict(U=fake, m=3, input=t, out=fake, n_out=4, amp=fake, prob=None, algo=0, param=0)
        a.update(kw)
        with pytest.raises(_abi.PcvError) as e:
            _abi.pcv_amplitudes_ex(a["U"], a["m"], a["input"], a["out"], a["n_out"], a["amp"], a["prob"],
                                   a["algo"], a["param"], None, 0, None)
        assert e.value.code == code, kw
    many = np.ones(40, np.uint8)
    with pytest.raises(_abi.PcvError) as e:
        _abi.pcv_amplitudes(fake, 40, many, fake, 1, fake, None, None, 0, None)
    assert e.value.code == _abi.PCV_EINVAL and "photons" in str(e.value)


def test_distribution_workspace_sizes():
    from paper_2204_00602_gb300 import _abi
    full = _abi.pcv_distribution_workspace(20, 10)
    small = _abi.pcv_distribution_workspace_min(20, 10)
    assert 0 < small < full < 8 << 30
    # the tensor-core plan: two real products per output, and 48 bytes of
    # digits per sign vector for each extension row (level n - 3 = 7 of the
    # ten modes of each side)
    N = math.comb(20 + 10 - 1, 10)
    rows = math.comb(10 + 7 - 1, 7)
    assert full >= 2 * N * 8 + 2 * rows * 512 * 48
    with pytest.raises(_abi.PcvError) as e:
        fake = 1 << 40
        _abi.pcv_distribution(fake, 20, np.array([1] * 10 + [0] * 10, np.uint8), fake, None, fake, small - 1024, None)
    assert e.value.code in (_abi.PCV_ENOMEM, _abi.PCV_EINVAL)


def test_explicit_algorithm_workspace_sizes():
    from paper_2204_00602_gb300 import _abi
    assert _abi.pcv_amplitudes_ex_workspace(20, 10, 100, _abi.PCV_ALGO_MULT, 1) == 0
    assert _abi.pcv_amplitudes_ex_workspace(20, 10, 100, _abi.PCV_ALGO_MULT, 4) >= 100 * 4 * 16
    # automatic warps per permanent: small output counts get several warps each
    assert _abi.pcv_amplitudes_ex_workspace(20, 10, 10, _abi.PCV_ALGO_MULT, 0) >= 10 * 2 * 16
    assert _abi.pcv_amplitudes_ex_workspace(20, 10, 1 << 20, _abi.PCV_ALGO_MULT, 0) == 0
    assert _abi.pcv_amplitudes_ex_workspace(20, 12, 100, _abi.PCV_ALGO_BLOCK, 2) >= 100 * 2 * 16
    assert _abi.pcv_amplitudes_ex_workspace(20, 10, 100, _abi.PCV_ALGO_AUTO, 0) == \
        _abi.pcv_amplitudes_workspace(20, 10, 100)
    with pytest.raises(_abi.PcvError) as e:
        _abi.pcv_amplitudes_ex_workspace(20, 10, 100, _abi.PCV_ALGO_MULT, 5000)
    assert e.value.code == _abi.PCV_EINVAL


def test_batched_routing_is_checked():
    from paper_2204_00602_gb300 import _abi
    fake = 1 << 40
    for algo in (_abi.PCV_ALGO_GROUP, _abi.PCV_ALGO_FACTOR, 99):
        with pytest.raises(_abi.PcvError) as e:
            _abi.pcv_amplitudes_batched_ex(fake, 2, 10, algo, fake, 1 << 20, None)
        assert e.value.code == _abi.PCV_EINVAL
    with pytest.raises(_abi.PcvError) as e:
        _abi.pcv_amplitudes_batched_ex(fake, 2, 1 << 31, _abi.PCV_ALGO_AUTO, fake, 1 << 40, None)
    assert e.value.code == _abi.PCV_ERANGE
    # the work lists grow with the outputs: three ints per output at least
    assert _abi.pcv_amplitudes_batched_workspace(4, 1000) >= 3 * 4 * 1000


def test_distinguishability_arguments_are_checked():
    from paper_2204_00602_gb300 import _abi
    fake = 1 << 40
    with pytest.raises(_abi.PcvError) as e:       # 17 photons: 2^17 pure sets is over the limit
        _abi.pcv_distribution_source(fake, 20, np.array([1] * 17 + [0] * 3, np.uint8), 1.0, 1.0, fake, fake,
                                     1 << 40, None)
    assert e.value.code == _abi.PCV_EINVAL
    for eta, V in ((1.2, 1.0), (0.5, -0.1), (float("nan"), 0.5)):
        with pytest.raises(_abi.PcvError) as e:
            _abi.pcv_distribution_source(fake, 4, np.array([1, 1, 0, 0], np.uint8), eta, V, fake, fake, 1 << 40, None)
        assert e.value.code == _abi.PCV_EINVAL
    cls = np.zeros((2, 4), np.uint8)
    cls[0, 0] = 20
    cls[1, 1] = 11                                 # 31 photons in all
    with pytest.raises(_abi.PcvError) as e:
        _abi.pcv_distribution_classes_workspace(4, 2, cls)
    assert e.value.code == _abi.PCV_EINVAL
    assert _abi.pcv_distribution_source_size(6, 3) == sum(math.comb(6 + k - 1, k) for k in range(4))
    cls[0, 0], cls[1, 1] = 2, 1
    assert _abi.pcv_distribution_classes_workspace(4, 2, cls) > 0


def test_tensor_core_workspace_sizes(lib):
    # host-only: the factorised tensor-core path's workspace (digit tensors of
    # the table levels 4..6 and the extension rows (level 7) of each side and
    # of the 3-photon column vectors, FP64 parents (levels 1..6), two products
    # per output, entry and seam data)
    from paper_2204_00602_gb300 import _abi
    ws = _abi.pcv_distribution_tc_workspace(20, 10)
    c = math.comb
    entries = sum(c(10 + k - 1, k) for k in (4, 5, 6, 7)) + c(20 + 3 - 1, 3)
    digits = 2 * entries * 3 * 8 * 512 * 2      # per side; 3 products x 8 digits x 512 sign vectors x 2 B
    parents = 2 * sum(c(10 + k - 1, k) for k in range(1, 7)) * 512 * 16
    products = 2 * c(29, 10) * 8
    assert digits + parents + products < ws < digits + parents + products + 0.1e9, ws
    assert _abi.pcv_distribution_tc_workspace(20, 9) < ws
    assert _abi.pcv_distribution_tc_workspace(12, 6) > 0
    with pytest.raises(_abi.PcvError):
        _abi.pcv_distribution_tc_workspace(20, 11)              # K = 2^{n-1} <= 512


def test_auto_algorithm_choice(lib):
    # host-only: pcv_distribution's AUTO takes the tensor-core products for
    # 2 <= n <= 10 when the workspace holds their plan, else the FP64 products
    from paper_2204_00602_gb300 import _abi
    tc = _abi.pcv_distribution_tc_workspace(20, 10)
    assert _abi.pcv_distribution_workspace(20, 10) == tc
    assert _abi.pcv_distribution_auto_algo(20, 10, tc) == _abi.PCV_ALGO_FACTOR_TC
    assert _abi.pcv_distribution_auto_algo(20, 10, tc - 1) == _abi.PCV_ALGO_FACTOR
    assert _abi.pcv_distribution_auto_algo(20, 11, 1 << 60) == _abi.PCV_ALGO_FACTOR
    assert _abi.pcv_distribution_auto_algo(20, 1, 1 << 60) == _abi.PCV_ALGO_FACTOR
    assert _abi.pcv_distribution_auto_algo(1, 4, 1 << 60) == _abi.PCV_ALGO_FACTOR
    assert _abi.pcv_distribution_auto_algo(12, 6, 1 << 40) == _abi.PCV_ALGO_FACTOR_TC
    assert _abi.pcv_distribution_workspace(20, 11) == _abi.pcv_distribution_batched_workspace(1, 20, 11)
    with pytest.raises(_abi.PcvError):
        _abi.pcv_distribution_auto_algo(0, 4, 0)


def test_static_entry_point_range_errors(lib):
    # host-only: an output space beyond int64 is a range error (as in
    # pcv_distribution), reported before any device work
    from paper_2204_00602_gb300 import _abi
    fake = 1 << 40
    with pytest.raises(_abi.PcvError) as e:
        _abi.pcv_distribution_static(fake, 1024, np.array([1] * 30 + [0] * 994, np.uint8), fake, fake, None)
    assert e.value.code == _abi.PCV_ERANGE


@pytest.mark.parametrize("m,n", [(7, 3), (6, 4), (9, 2), (2, 3), (1, 3), (5, 5)])
def test_range_plan_against_enumeration(lib, m, n):
    # host-only: for ranges of the canonical order, the low-side multisets P
    # (photons in modes [0, h), ranked at their size k) that the range
    # computes are exactly those of the outputs inside it, found here by
    # walking itertools' enumeration of S_{m,n}
    from paper_2204_00602_gb300 import _abi
    h = max(1, m // 2)
    outs = list(itertools.combinations_with_replacement(range(m), n))
    rank_of = {k: {P: i for i, P in enumerate(itertools.combinations_with_replacement(range(h), k))}
               for k in range(n + 1)}
    N = len(outs)
    cuts = sorted({0, 1, N // 3, N // 2, N - 1, N, 5 % (N + 1), (7 * N) // 11})
    ranges = [(a, b) for a in cuts for b in cuts if a <= b]
    for begin, end in ranges:
        want = [[None, None] for _ in range(n + 1)]
        for S in outs[begin:end]:
            P = tuple(x for x in S if x < h)
            r = rank_of[len(P)][P]
            w = want[len(P)]
            w[0] = r if w[0] is None else min(w[0], r)
            w[1] = r + 1 if w[1] is None else max(w[1], r + 1)
        got = _abi.pcv_distribution_range_plan(m, n, begin, end)
        for k in range(n + 1):
            a, b = got[k]
            if want[k][0] is None:
                assert a >= b, (begin, end, k, got[k])
            else:
                assert (a, b) == tuple(want[k]), (begin, end, k, got[k], want[k])
    with pytest.raises(_abi.PcvError):
        _abi.pcv_distribution_range_plan(m, n, 0, N + 1)


def test_tc_block_view_errors(lib):
    # host-only: sizes outside the tensor-core plan, a bad range and a short
    # output array are argument errors; end < 0 means the whole space
    import ctypes
    from paper_2204_00602_gb300 import _abi
    for m, n in ((1, 4), (6, 1), (6, 11), (1025, 3)):
        with pytest.raises(_abi.PcvError) as e:
            _abi.pcv_distribution_tc_blocks(m, n)
        assert e.value.code == _abi.PCV_EINVAL
    N = _abi.pcv_num_outputs(7, 4)
    for begin, end in ((-1, 5), (6, 5), (0, N + 1)):
        with pytest.raises(_abi.PcvError) as e:
            _abi.pcv_distribution_tc_blocks(7, 4, begin, end)
        assert e.value.code == _abi.PCV_EINVAL
    f = _abi._lib.pcv_distribution_tc_blocks          # argument types set by the binding
    need = ctypes.c_int64(0)
    assert f(7, 4, 0, -1, None, 0, ctypes.addressof(need)) == 0
    out = (ctypes.c_int64 * need.value)()
    assert f(7, 4, 0, -1, ctypes.addressof(out), need.value - 1, None) == _abi.PCV_EINVAL
    assert f(7, 4, 0, N, ctypes.addressof(out), need.value, None) == 0
    assert out[3] >= 1 and need.value - 48 == 16 * out[3]
