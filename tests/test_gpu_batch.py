"""Batched classification (one persistent launch over uneven frames) gives
exactly the per-frame results, also when replayed from a captured CUDA graph."""
import numpy as np
import pytest

import oracle as O
from paper_1603_05143_gb300 import inputs as I
from parity import compare

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


def _dev(frames):
    import torch
    return [{"positions": torch.from_numpy(np.ascontiguousarray(f.positions)).cuda(),
             "species": torch.from_numpy(f.species.astype(np.int8)).cuda(), "cell": f.cell, "pbc": f.pbc}
            for f in frames]


def _np(o):
    return {k: v.cpu().numpy() for k, v in o.items()}


def test_batch_equals_single_frames(ptm):
    import torch
    frames = I.config_batch(seed=31, n_frames=14, n_min=200, n_max=30000)
    dev = _dev(frames)
    b = ptm.batch(dev)
    b.run()
    torch.cuda.synchronize()
    st = b.stats()
    assert st["internal"] == 0 and st["atoms"] == sum(f.n for f in frames)
    for f, d, o in zip(frames, dev, b.outputs):
        ref = ptm.classify(d["positions"], f.cell, f.pbc, species=d["species"])
        torch.cuda.synchronize()
        for k in ref:
            assert torch.equal(ref[k], o[k]), (f.name, k)
    # two frames checked against the oracle as well
    for f, o in list(zip(frames, b.outputs))[:2]:
        atoms = np.arange(0, f.n, max(1, f.n // 300))
        ref = O.classify_frame(f, atoms=atoms)
        compare(_np(o), ref, atoms)
    b.close()


@pytest.mark.parametrize("tile", [32, 64, 96])
def test_batch_with_large_frames_and_tiles(ptm, tile):
    """Frames of 65536 atoms or more take their own matching launch, the
    others the shared persistent one; tiles of 64 and 96 slots leave chunks
    past the end of the atoms: every frame still equals its single-frame
    result."""
    import torch
    frames = I.config_batch(seed=12, n_frames=5, n_min=300, n_max=3000)
    frames.insert(2, I.crystal("bcc", I.A_BCC_FE, 33, sigma=0.1, seed=4, dtype=np.float32,
                               rotation=I.random_rotation(I.rng_for(6))))        # 71874 atoms
    frames.append(I.crystal("fcc", I.A_FCC_CU, 26, sigma=0.12, seed=5, dtype=np.float32))   # 70304 atoms
    dev = _dev(frames)
    b = ptm.batch(dev, tuning={"tile_atoms": tile})
    b.run()
    torch.cuda.synchronize()
    st = b.stats()
    assert st["internal"] == 0 and st["atoms"] == sum(f.n for f in frames)
    assert st["kernel_launches"] == 8 + 2                 # two frames with their own k_match
    for f, d, o in zip(frames, dev, b.outputs):
        ref = ptm.classify(d["positions"], f.cell, f.pbc, species=d["species"])
        torch.cuda.synchronize()
        for k in ref:
            assert torch.equal(ref[k], o[k]), (f.name, k)
    b.close()


def test_batch_graph_replay_follows_positions(ptm):
    import torch
    frames = I.config_batch(seed=7, n_frames=6, n_min=500, n_max=5000)
    dev = _dev(frames)
    s = torch.cuda.Stream()
    b = ptm.batch(dev, tuning={"cell_factor": 1.4, "tile_atoms": 64})
    with torch.cuda.stream(s):
        b.run(s)
        s.synchronize()
        first = [_np(o) for o in b.outputs]
        b.capture(s)
        b.run(s)
        s.synchronize()
    st = b.stats()                       # events recorded by the graph replay
    assert st["atoms"] == sum(f.n for f in frames) and st["atom_kernel_ms"] > 0
    for a, o in zip(first, b.outputs):
        for k in a:
            assert np.array_equal(a[k], o[k].cpu().numpy()), k
    # new positions in place (next MD frame), replay the graph
    rng = np.random.default_rng(3)
    for f, d in zip(frames, dev):
        f.positions = (f.positions + rng.normal(0, 0.05, f.positions.shape)).astype(np.float32)
        d["positions"].copy_(torch.from_numpy(f.positions))
    with torch.cuda.stream(s):
        b.run(s)
        s.synchronize()
    for f, d, o in zip(frames, dev, b.outputs):
        ref = ptm.classify(d["positions"], f.cell, f.pbc, species=d["species"])
        torch.cuda.synchronize()
        for k in ref:
            assert torch.equal(ref[k], o[k]), k
    b.close()


def test_autotune_returns_valid_tuning(ptm, tmp_path):
    frames = I.config_batch(seed=5, n_frames=4, n_min=1000, n_max=4000)
    dev = _dev(frames)
    cache = str(tmp_path / "tuning.json")
    t = ptm.autotune(dev, cache=cache)
    assert t["cell_factor"] in (1.125, 1.25, 1.4)
    assert t["tile_atoms"] in (32, 64) and t["blocks_per_sm"] in (7, 8)
    assert ptm.autotune(dev, cache=cache) == t           # served from the cache
