"""The allocation-free table build agrees with the regular one.

hq_dispatch_table_static serves callers that may not allocate device memory (an
external pool or a fixed budget owns every buffer, or a cudaMalloc's device-wide
synchronisation is not acceptable): its working memory is a fixed static device
array.  This file is collected last on purpose, so a failure here comes after every
other test has run.
"""
import math

import numpy as np
import pytest

from paper_2603_03019_gb300 import hq
from paper_2603_03019_gb300 import instances as I

pytestmark = pytest.mark.gpu


def _regular_table(inst):
    s = hq.Solver.for_instance(inst)
    T, _ = s.table()
    s.close()
    return T


def test_static_table_matches_regular_entry_point_twice(gpu_lib):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    # two calls in a row: the second (smaller N, more nodes) must not see the
    # first call's leftovers in the shared static array
    cases = [I.geometric_instance(14, 300, 71, 0.7, nu_lo=0.5, nu_hi=1.5),
             I.geometric_instance(11, 1500, 72, 0.7, nu_lo=0.5, nu_hi=1.5)]
    for inst in cases:
        lam = torch.tensor(inst.lam_j, device=dev)
        pref = torch.tensor(inst.pref, device=dev)
        T = torch.full((inst.N << (inst.N - 1),), float("nan"), dtype=torch.float64, device=dev)
        hq.hq_dispatch_table_static(inst.N, inst.J, lam, pref, T, stream)
        torch.cuda.synchronize()
        got = T.cpu().numpy()
        want = _regular_table(inst)
        assert got.shape == want.shape
        # both builds quantise every rate to the same 64-bit fixed point and add integers,
        # so the tables agree bit for bit
        assert np.array_equal(got, want)


def test_static_table_rejects_oversize_and_bad_rows(gpu_lib):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    lam = torch.ones(4, dtype=torch.float64, device=dev)
    pref = torch.zeros((4, 17), dtype=torch.int32, device=dev)
    T = torch.zeros(17 << 16, dtype=torch.float64, device=dev)
    # sizes beyond the static array are refused by the C entry point itself, before it
    # touches any pointer (called directly: the binding would stop the short tensors first)
    lib = hq.load()
    for N, J in ((17, 4), (8, 5000)):
        rc = lib.hq_dispatch_table_static(N, J, lam.data_ptr(), pref.data_ptr(), T.data_ptr(), None)
        assert rc == hq.HQ_EINVAL
    # the binding checks what the C side cannot: dtype, device, contiguity and length
    with pytest.raises(ValueError):
        hq.hq_dispatch_table_static(8, 5000, lam, pref, T)
    with pytest.raises(ValueError):
        hq.hq_dispatch_table_static(4, 4, lam.float(), pref, T)
    bad = torch.zeros((4, 6), dtype=torch.int32, device=dev)  # rows are not permutations
    with pytest.raises(hq.HQError) as e:
        hq.hq_dispatch_table_static(6, 4, lam, bad, T)
    assert e.value.code == hq.HQ_EINVAL
    assert math.isfinite(float(T[0]))
