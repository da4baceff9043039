"""Serving: frames submitted while others run give exactly the results they
give alone (continuous batching), under an HBM budget (GPU only)."""
import time

import numpy as np
import pytest

from paper_1603_05143_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ptm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_05143_gb300 import PTM
    p = PTM(0)
    yield p
    p.close()


def _frames():
    fr = I.config_batch(seed=41, n_frames=10, n_min=500, n_max=60000)
    fr.append(I.config_fcc_small())          # float64 frame: served in a batch of its own dtype
    return fr


def test_alone_equals_in_the_mix(ptm):
    from paper_1603_05143_gb300 import Server
    frames = _frames()
    srv = Server(ptm, streams=2, max_batch_frames=8)
    alone = []
    for f in frames:                         # one at a time
        t = srv.submit(f.positions, f.cell, f.pbc, species=f.species)
        alone.append({k: v.copy() for k, v in srv.wait(t, 60000).items()})
        srv.release(t)
    rng = np.random.default_rng(0)
    order = rng.permutation(len(frames))
    for burst in (False, True):              # staggered arrivals, then all at once
        tickets = {}
        for i in order:
            f = frames[i]
            tickets[i] = srv.submit(f.positions, f.cell, f.pbc, species=f.species, pinned=True)
            if not burst:
                time.sleep(float(rng.uniform(0, 0.002)))
        batches = set()
        for i, t in tickets.items():
            out = srv.wait(t, 60000)
            info = srv.info(t)
            assert info["submit"] <= info["start"] <= info["done"]
            batches.add(info["batch"])
            for k in out:
                assert np.array_equal(out[k], alone[i][k]), (frames[i].name, k, burst)
            srv.release(t)
        if burst:
            assert len(batches) < len(frames)    # queued frames shared launches
    # and the device entry point agrees
    import torch
    f = frames[3]
    ref = ptm.classify(torch.from_numpy(f.positions).cuda(), f.cell, f.pbc,
                       species=torch.from_numpy(f.species).cuda())
    torch.cuda.synchronize()
    for k in ref:
        assert np.array_equal(ref[k].cpu().numpy(), alone[3][k]), k
    srv.close()


def test_budget_admission_and_errors(ptm):
    from paper_1603_05143_gb300 import PTMError, Server
    frames = I.config_batch(seed=42, n_frames=6, n_min=2000, n_max=8000)
    biggest = max(f.n for f in frames)
    srv = Server(ptm, hbm_budget_bytes=400 * biggest, streams=2)   # room for about one frame at a time
    ts = [srv.submit(f.positions, f.cell, f.pbc, species=f.species) for f in frames]
    for t in ts:
        srv.wait(t, 60000)
    infos = [srv.info(t) for t in ts]
    starts = [i["start"] for i in infos]
    assert starts == sorted(starts)                  # admitted in arrival order
    # a frame over the budget is refused, never launched
    big = I.crystal("fcc", I.A_FCC_CU, 24, sigma=0.05, seed=1, dtype=np.float32)     # 55296 atoms
    assert big.n * 250 > 400 * biggest
    t = srv.submit(big.positions, big.cell, big.pbc)
    with pytest.raises(PTMError) as e:
        srv.wait(t, 60000)
    assert "OUT_OF_MEMORY" in str(e.value)
    with pytest.raises(PTMError) as e:
        srv.wait(123456789, 10)
    assert "NOT_FOUND" in str(e.value)
    srv.close()


def test_wait_times_out_then_completes(ptm):
    from paper_1603_05143_gb300 import PTMError, Server
    f = I.crystal("bcc", I.A_BCC_FE, 40, sigma=0.1, seed=2, dtype=np.float32)     # 128000 atoms
    srv = Server(ptm)
    t = srv.submit(f.positions, f.cell, f.pbc)
    try:
        srv.wait(t, 0)
        timed_out = False
    except PTMError as e:
        timed_out = "TIMEOUT" in str(e)
    out = srv.wait(t, 60000)
    assert (out["structure"] == 5).mean() > 0.9
    assert timed_out or srv.poll(t)
    srv.close()
