"""The Python binding's argument checks, on the CPU, against a stub of libhq.so.

The C side receives bare pointers and cannot check what they point to, so the binding
checks every buffer before the call: element type, C-contiguity, at least the number of
elements the call writes or reads (from the solver's sizes), and for CUDA tensors the
current device.  A rejected buffer raises ValueError and no C call is made.  A buffer the
binding converts (warm_p of another type) stays alive through the call.
"""
import ctypes

import numpy as np
import pytest

from paper_2603_03019_gb300 import hq

N, J, C = 4, 3, 2


class StubLib:
    """Records each call; hq_get_info reports a solver of N units, J nodes, finite
    buffer C; hq_solve reads the warm start it is given."""

    def __init__(self):
        self.calls = []
        self.warm_seen = None

    def hq_get_info(self, h, addr):
        out = (ctypes.c_int64 * 8).from_address(addr)
        out[:] = [N, J, hq.HQ_FINITE, C, 1 << N, N << (N - 1), 0, 0]
        return 0

    def hq_solve(self, h, opts, stats):
        o = opts._obj
        if o.warm_p:
            self.warm_seen = np.ctypeslib.as_array((ctypes.c_double * (1 << N)).from_address(o.warm_p)).copy()
        self.calls.append(("hq_solve",))
        return 0

    def hq_default_opts(self, ref):
        return None

    def hq_strerror(self, rc):
        return b"stub"

    def hq_last_error(self):
        return b"stub"

    def hq_mlp_num_params(self, m):
        return 10

    def __getattr__(self, name):
        def call(*args):
            self.calls.append((name,) + args)
            return 0
        return call


@pytest.fixture()
def stub(monkeypatch):
    lib = StubLib()
    monkeypatch.setattr(hq, "_lib", lib)
    return lib


def _names(lib):
    return [c[0] for c in lib.calls]


def test_load_passes_checked_buffers(stub):
    lam, nu, pref = np.ones(J), np.ones(N), np.zeros((J, N), np.int32)
    hq.hq_load(7, lam, nu, pref)
    assert stub.calls == [("hq_load", 7, lam.ctypes.data, nu.ctypes.data, pref.ctypes.data, hq.HQ_HOST)]


@pytest.mark.parametrize("bad", ["lam_type", "nu_short", "pref_type", "pref_strided", "torch_type"])
def test_load_rejects_bad_buffers_before_the_call(stub, bad):
    import torch

    lam, nu, pref = np.ones(J), np.ones(N), np.zeros((J, N), np.int32)
    if bad == "lam_type":
        lam = lam.astype(np.float32)
    elif bad == "nu_short":
        nu = nu[:-1]
    elif bad == "pref_type":
        pref = pref.astype(np.int64)
    elif bad == "pref_strided":
        pref = np.zeros((J, 2 * N), np.int32)[:, ::2]
    else:
        lam = torch.ones(J, dtype=torch.float32)
    with pytest.raises(ValueError):
        hq.hq_load(7, lam, nu, pref)
    assert "hq_load" not in _names(stub)


def test_getters_check_output_sizes(stub):
    hq.hq_get_stationary(1, np.empty(1 << N))
    hq.hq_get_response_pattern(1, np.empty((J, N)))
    hq.hq_get_workload(1, np.empty((N, J)))
    hq.hq_get_utilisation(1, np.empty(N))
    # finite buffer: p(0..N+C)
    hq.hq_get_layer_marginals(1, np.empty(N + C + 1), np.zeros(1))
    n_ok = len(stub.calls)
    for fn, out in ((hq.hq_get_stationary, np.empty((1 << N) - 1)), (hq.hq_get_conditional, np.empty(3)),
                    (hq.hq_get_response_pattern, np.empty((J, N - 1))), (hq.hq_get_utilisation, np.empty(N, np.float32)),
                    (hq.hq_get_layer_marginals, np.empty(N + 1))):
        with pytest.raises(ValueError):
            fn(1, out)
    assert len(stub.calls) == n_ok


def test_table_masks_take_either_32_bit_type(stub):
    T = np.empty(N << (N - 1))
    hq.hq_get_table(1, T, np.empty(1 << N, np.uint32))
    hq.hq_get_table(1, T, np.empty(1 << N, np.int32))
    assert _names(stub).count("hq_get_table") == 2
    with pytest.raises(ValueError):
        hq.hq_get_table(1, T, np.empty(1 << N, np.float32))
    with pytest.raises(ValueError):
        hq.hq_get_table(1, np.empty(5), None)


def test_torch_host_tensors_are_host_memory(stub):
    import torch

    out = torch.empty(1 << N, dtype=torch.float64)
    hq.hq_get_stationary(1, out)
    assert stub.calls[-1] == ("hq_get_stationary", 1, out.data_ptr(), hq.HQ_HOST)
    with pytest.raises(ValueError):
        hq.hq_get_stationary(1, torch.empty(1 << N, dtype=torch.float32))


def test_converted_warm_start_lives_through_the_call(stub):
    s = hq.Solver.__new__(hq.Solver)
    s.h, s.N, s.J, s.mode, s.C = 1, N, J, hq.HQ_FINITE, C
    warm = np.arange(1 << N, dtype=np.float32) / 16
    s.solve(warm_p=warm)
    assert np.array_equal(stub.warm_seen, warm.astype(np.float64))
    with pytest.raises(ValueError):
        s.solve(warm_p=np.ones((1 << N) - 1))


def test_mlp_buffers(stub):
    hq.hq_mlp_set_weights(3, np.zeros(10, np.float32))
    with pytest.raises(ValueError):
        hq.hq_mlp_set_weights(3, np.zeros(9, np.float32))
    with pytest.raises(ValueError):
        hq.hq_mlp_set_weights(3, np.zeros(10))
    X = hq.hq_mlp_features(1)
    assert X.shape == (N * (N - 1), 9)
    with pytest.raises(ValueError):
        hq.hq_mlp_features(1, N=N + 1)
    with pytest.raises(ValueError):
        # network inputs must be CUDA tensors
        hq.hq_mlp_forward(3, np.zeros((5, 9), np.float32), np.zeros(5, np.float32))


def test_simulation_inputs(stub):
    lam, nu, pref, tt = np.ones(J), np.ones(N), np.zeros((J, N), np.int32), np.ones((J, N))
    hq.hq_des_simulate(N, J, lam, nu, pref, tt, "gamma5", 6, 100, 10, 1)
    call = stub.calls[-1]
    assert call[0] == "hq_des_simulate" and call[1:3] == (N, J) and call[-2] == hq.HQ_HOST
    with pytest.raises(ValueError):
        hq.hq_des_simulate(N, J, lam, nu, pref, np.ones((J, N - 1)), "gamma5", 6, 100, 10, 1)
