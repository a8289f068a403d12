"""The allocation-free binning entry point, called through the C ABI.

tred_blockbin_noalloc serves callers that cannot allocate device memory once they
run (a host framework that owns all device memory through its own pool, or a
real-time loop that cannot afford the synchronisation of cudaMalloc).  It must give
what tred_blockbin gives on the same inputs, call after call, although every call
reuses the same static scratch.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _bin_both(cfg, dep, mb=None):
    import torch
    from paper_2602_12052_b300 import abi, build, tred
    build.build()
    lib = abi.load()
    dev = torch.device("cuda")
    n = len(dep["x"])
    mb = mb or min(cfg.n_blocks, 20000)
    h = tred.Handle(tred.geometry(cfg), tred.params(cfg), max(n, 1), mb, 1)
    deps = tred.DepositBuffers(max(n, 1), dev)
    x = {k: torch.from_numpy(v).to(dev) for k, v in dep.items()}
    if n:
        tred.tred_drift(h, n, x["x"], x["y"], x["z"], x["t0"], x["ne"], deps)
    mp = 8 * max(n, 1)

    def bufs():
        return (torch.zeros(mb, dtype=torch.int32, device=dev), torch.zeros(mb, dtype=torch.int32, device=dev),
                torch.zeros(mb + 1, dtype=torch.int32, device=dev), torch.zeros(mp, dtype=torch.int32, device=dev),
                torch.zeros(1, dtype=torch.int32, device=dev))

    ref = bufs()
    tred.tred_blockbin(h, n, deps, *ref[:4], ref[4])
    ref_status = tred.tred_sync_status(h)
    outs = []
    geom = tred.geometry(cfg)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):                       # two calls in a row share the static scratch
        o = bufs()
        status = torch.zeros(8, dtype=torch.int32, device=dev)
        rc = lib.tred_blockbin_noalloc(ctypes.byref(geom), n, ctypes.byref(deps.struct),
                                       *(ctypes.c_void_p(t.data_ptr()) for t in o[:4]), mb, mp,
                                       ctypes.c_void_p(o[4].data_ptr()), ctypes.c_void_p(status.data_ptr()),
                                       stream)
        assert rc == abi.TRED_OK
        torch.cuda.synchronize()
        outs.append((o, status.cpu().numpy()))
    return ref, ref_status, outs


def _same(ref, o):
    nb = int(ref[4].item())
    assert int(o[4].item()) == nb
    for a, b in zip(ref[:2], o[:2]):
        np.testing.assert_array_equal(a[:nb].cpu().numpy(), b[:nb].cpu().numpy())
    off = ref[2][:nb + 1].cpu().numpy()
    np.testing.assert_array_equal(off, o[2][:nb + 1].cpu().numpy())
    # CSR: the same deposit ids in the same (ascending per block) order, which fixes the
    # order of the effective charge's sums downstream
    ri, oi = ref[3].cpu().numpy(), o[3].cpu().numpy()
    np.testing.assert_array_equal(ri[:off[nb]], oi[:off[nb]])
    return nb


@pytest.mark.parametrize("name", ["tiny", "module200"])
def test_noalloc_blockbin_matches_handle_path(name):
    cfg = synth.get_config(name)
    dep = synth.make_deposits(cfg)
    ref, ref_status, outs = _bin_both(cfg, dep)
    for o, status in outs:
        nb = _same(ref, o)
        assert nb > 0
        assert status[0] == ref_status[0] == 0
        assert status[2] == ref_status[2] and status[3] == ref_status[3]


def test_noalloc_blockbin_empty_event():
    """No deposits: no blocks, an empty CSR and a clear status, call after call."""
    cfg = synth.get_config("tiny")
    dep = {k: np.zeros(0, np.float32) for k in ("x", "y", "z", "t0", "ne")}
    ref, ref_status, outs = _bin_both(cfg, dep)
    for o, status in outs:
        assert _same(ref, o) == 0
        assert int(o[2][0].item()) == 0
        assert status[0] == ref_status[0] == 0 and status[2] == 0 and status[3] == 0


def test_noalloc_blockbin_block_overflow_matches_handle_path():
    """max_blocks below the event's active block count: both paths set the block-overflow
    bit, keep the first max_blocks blocks in order and clamp the CSR the same way."""
    from paper_2602_12052_b300 import abi
    cfg = synth.get_config("tiny")
    dep = synth.make_deposits(cfg)
    ref, ref_status, outs = _bin_both(cfg, dep, mb=3)
    assert ref_status[2] > 3                 # more active blocks than kept
    for o, status in outs:
        assert _same(ref, o) == 3
        assert status[0] & abi.TRED_ST_BLOCK_OVERFLOW
        assert status[0] == ref_status[0]
        assert status[2] == ref_status[2] and status[3] == ref_status[3]


def test_noalloc_rejects_oversized_plane():
    from paper_2602_12052_b300 import abi, build, tred
    build.build()
    lib = abi.load()
    cfg = synth.get_config("tiny", npx=2048, nt=65536, bt=64)   # 256*256*1024 blocks
    geom = tred.geometry(cfg)
    rc = lib.tred_blockbin_noalloc(ctypes.byref(geom), 0, None, *([ctypes.c_void_p(16)] * 4), 10, 10,
                                   ctypes.c_void_p(16), ctypes.c_void_p(16), None)
    assert rc == abi.TRED_ERR_CAPACITY
