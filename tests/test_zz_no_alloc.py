"""genga_kick_noalloc, the kick phase for callers that cannot allocate device memory.

Such callers (a latency-critical loop, where cudaFree would synchronise the device, or a host
framework that owns the device memory) call this entry point instead of genga_phase_kick. It
must give the same accelerations and candidate list as genga_phase_kick, on consecutive calls
that reuse its one static scratch array. This file sorts last so that a run stopping at the
first failure has already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1404_2324_gb300 import genga, ics
from tests.gpu_util import aos, dev, soa, torch

pytestmark = pytest.mark.gpu


def _inputs(n, seed):
    d = ics.disk2048(seed)
    p = O.params(G=d["G"], m0=d["m0"], dt=d["dt"])
    sel = np.sort(np.random.default_rng(seed).choice(2048, n, replace=False))
    m, x, v = d["m"][sel], d["x"][sel], d["v"][sel]
    alive = np.ones(n, np.int32)
    alive[3] = 0
    rc = O.rcrit(p, 6.0, m, alive, x, v) * 6.0  # many near pairs
    return d["G"], m, alive, x, rc


def test_noalloc_kick_matches_allocating_kick_on_two_calls():
    L = genga.lib()
    stream = torch().cuda.current_stream()
    for call, (n, seed) in enumerate(((1024, 21), (700, 22))):
        G, m, alive, x, rc = _inputs(n, seed)
        cap = n * (n - 1) // 2
        a_ref, c_ref = dev(np.zeros((3, n))), dev(np.zeros(2 * cap, np.int32))
        nref = genga.genga_phase_kick(n, G, 3.0, 0, 0, dev(m), dev(alive), soa(x), dev(rc), a_ref, c_ref, cap)
        a, cand, cnt = dev(np.zeros((3, n))), dev(np.zeros(2 * cap, np.int32)), dev(np.zeros(1, np.int32))
        V = ctypes.c_void_p
        ms, als, xs, rcs = dev(m), dev(alive), soa(x), dev(rc)
        rc_ = L.genga_kick_noalloc(n, G, 3.0, 0, 0, V(ms.data_ptr()), V(als.data_ptr()), V(xs.data_ptr()),
                                   V(rcs.data_ptr()), V(a.data_ptr()), V(cand.data_ptr()), cap, V(cnt.data_ptr()),
                                   V(stream.cuda_stream))
        assert rc_ == 0, (call, rc_)
        torch().cuda.synchronize()
        k = int(cnt.item())
        assert k == nref and k > 0, call
        np.testing.assert_array_equal(cand.cpu().numpy()[: 2 * k], c_ref.cpu().numpy()[: 2 * k])
        ga, ra = aos(a), aos(a_ref)
        np.testing.assert_allclose(ga, ra, rtol=0, atol=1e-13 * np.abs(ra).max())


def test_noalloc_kick_rejects_sizes_above_its_maximum():
    L = genga.lib()
    V = ctypes.c_void_p
    z = dev(np.zeros(8))
    assert L.genga_kick_noalloc(1025, 1.0, 3.0, 0, 0, V(z.data_ptr()), V(z.data_ptr()), V(z.data_ptr()),
                                V(z.data_ptr()), V(z.data_ptr()), V(z.data_ptr()), 1, V(z.data_ptr()),
                                None) == genga.GENGA_ESIZE


def test_noalloc_kick_with_a_small_cap_reports_the_full_count():
    """cap below the candidate count: *ncand (on the device) is the full count, the first cap pairs
    are the allocating kick's first cap pairs, and no device memory changes hands across calls."""
    L = genga.lib()
    V = ctypes.c_void_p
    stream = torch().cuda.current_stream()
    n, seed = 512, 23
    G, m, alive, x, rc = _inputs(n, seed)
    full = n * (n - 1) // 2
    a_ref, c_ref = dev(np.zeros((3, n))), dev(np.zeros(2 * full, np.int32))
    nref = genga.genga_phase_kick(n, G, 3.0, 0, 0, dev(m), dev(alive), soa(x), dev(rc), a_ref, c_ref, full)
    cap = nref // 3
    assert cap > 0
    ms, als, xs, rcs = dev(m), dev(alive), soa(x), dev(rc)
    a, cand, cnt = dev(np.zeros((3, n))), dev(np.zeros(2 * cap, np.int32)), dev(np.zeros(1, np.int32))

    def call():
        return L.genga_kick_noalloc(n, G, 3.0, 0, 0, V(ms.data_ptr()), V(als.data_ptr()), V(xs.data_ptr()),
                                    V(rcs.data_ptr()), V(a.data_ptr()), V(cand.data_ptr()), cap, V(cnt.data_ptr()),
                                    V(stream.cuda_stream))

    assert call() == 0
    torch().cuda.synchronize()
    free0 = torch().cuda.mem_get_info()[0]
    for _ in range(2):
        assert call() == 0
        torch().cuda.synchronize()
    assert torch().cuda.mem_get_info()[0] == free0
    assert int(cnt.item()) == nref
    np.testing.assert_array_equal(cand.cpu().numpy(), c_ref.cpu().numpy()[: 2 * cap])
