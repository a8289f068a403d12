"""The streaming entry point (tred.StreamRunner): host-resident events through one
Simulator with the input copies and the result read-back on side streams, overlapped with
the neighbouring events' steps.  Each event's counts and hit list equal those of the same
event run alone through Simulator.step, bit for bit (the step's sums have a fixed order),
whatever the queue's state."""
import numpy as np
import pytest

import synth
from parity_util import make_sim, to_dev

pytestmark = pytest.mark.gpu


def _events(cfg):
    sizes = [500, 37, 0, 260, 1, 499]
    out = []
    for i, m in enumerate(sizes):
        dep = synth.make_deposits(cfg, seed=cfg.seed + 1000 * i)
        out.append({k: v[:m].copy() for k, v in dep.items()})
    return out


@pytest.mark.parametrize("conv_mode,fuse", [(4, True), (4, False), (0, False)])
def test_stream_runner_equals_single_steps(conv_mode, fuse):
    import torch
    from paper_2602_12052_b300 import tred
    cfg = synth.get_config("tiny")
    resp = synth.make_response(cfg)
    events = _events(cfg)
    cap = max(len(e["x"]) for e in events)
    sim = make_sim(cfg, resp, cap, conv_mode=conv_mode, effq_skip_empty=1 if conv_mode == 4 else 0,
                   fuse_gather=fuse)
    runner = tred.StreamRunner(sim, cap)
    got = []
    for k, dep in enumerate(events):
        host = {f: torch.from_numpy(np.ascontiguousarray(dep[f])).pin_memory() for f in runner.FIELDS}
        r = runner.submit(host, len(dep["x"]), tag=k)
        if r is not None:
            got.append(r)
    got += runner.drain()
    assert [t for t, _ in got] == list(range(len(events)))
    assert sim.status()[0] == 0
    for k, dep in enumerate(events):
        n = len(dep["x"])
        t = to_dev(dep)
        sim.step(n, t["x"], t["y"], t["z"], t["t0"], t["ne"])
        ref = sim.results()
        res = got[k][1]
        assert (res["n_blocks"], res["n_pixels"], res["n_hits"]) == (ref["n_blocks"], ref["n_pixels"], ref["n_hits"])
        for key in ("hit_pixel", "hit_tick", "hit_charge"):
            np.testing.assert_array_equal(res[key], ref[key])
        if n == 0:
            assert res["n_blocks"] == 0 and res["n_hits"] == 0
