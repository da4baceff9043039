"""Fault handling (GPU only; no GPU fault is ever caused): atoms with
non-finite or far-away coordinates, a serving batch whose completion goes
unseen or fails (injected on the host), and frames re-submitted to a new
context and server after the first ones were destroyed."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1603_05143_gb300 import inputs as I
from parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def ptm(torch):
    from paper_1603_05143_gb300 import PTM
    p = PTM(0)
    yield p
    p.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_nonfinite_and_far_atoms_are_excluded(ptm, torch, dtype):
    """Atoms with a NaN or infinite coordinate, or 1000 periods from the cell,
    come out unmatched (structure NONE, the unmatched outputs), are counted in
    the excluded statistic, and are nobody's neighbour: every other atom gets
    the oracle's answer on the frame without them."""
    f = I.crystal("fcc", I.A_FCC_CU, 5, sigma=0.08, seed=12, dtype=np.float64,
                  rotation=I.random_rotation(I.rng_for(13)))
    pos = f.positions.copy()
    bad = np.array([3, 77, 150, 301, 402])
    pos[bad[0], 0] = np.nan
    pos[bad[1], 1] = np.inf
    pos[bad[2], 2] = -np.inf
    pos[bad[3]] = pos[bad[3]] + 1000.0 * f.cell[0]
    pos[bad[4], :] = np.nan
    pos = pos.astype(dtype)
    out = ptm.classify(torch.from_numpy(pos).cuda(), f.cell, f.pbc)
    torch.cuda.synchronize()
    st = ptm.stats()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    assert st["excluded"] == len(bad) and st["internal"] == 0
    assert np.all(g["structure"][bad] == 0) and np.all(np.isinf(g["rmsd"][bad]))
    assert np.all(g["correspondence"][bad] == -1)
    keep = np.setdiff1d(np.arange(f.n), bad)
    clean = I.Frame(pos[keep], f.cell, f.pbc, None, "clean")
    ref = O.Frame(clean.positions, clean.cell, clean.pbc).classify(None)
    # the GPU frame's atom ids -> ids of the clean frame, for the correspondence
    remap = -np.ones(f.n, np.int64)
    remap[keep] = np.arange(len(keep))
    gk = {k: v[keep] for k, v in g.items()}
    gk["correspondence"] = np.where(gk["correspondence"] >= 0, remap[np.maximum(gk["correspondence"], 0)], -1)
    compare(gk, ref)


def _frames():
    return I.config_batch(seed=77, n_frames=6, n_min=800, n_max=20000)


def _reference(ptm, torch, frames):
    ref = []
    for f in frames:
        out = ptm.classify(torch.from_numpy(f.positions).cuda(), f.cell, f.pbc,
                           species=torch.from_numpy(f.species).cuda())
        torch.cuda.synchronize()
        ref.append({k: v.cpu().numpy() for k, v in out.items()})
    return ref


def _equal(out, ref):
    for k in ref:
        assert np.array_equal(out[k], ref[k]), k


def test_lost_completion_times_out_then_recovers(ptm, torch):
    """The completion of one batch goes unseen (injected on the host): waits
    on its ticket time out and it stays not done, while a frame submitted
    afterwards completes on the other stream; once the completion is seen
    again the held frame finishes with the right outputs."""
    from paper_1603_05143_gb300 import PTMError, Server
    frames = _frames()[:2]
    ref = _reference(ptm, torch, frames)
    srv = Server(ptm, streams=2, max_batch_frames=1)
    srv.inject("hold_next")
    ta = srv.submit(frames[0].positions, frames[0].cell, frames[0].pbc, species=frames[0].species)
    with pytest.raises(PTMError) as e:
        srv.wait(ta, timeout_ms=300)
    assert e.value.status == 4                        # PTM_ERR_TIMEOUT
    assert not srv.poll(ta)
    tb = srv.submit(frames[1].positions, frames[1].cell, frames[1].pbc, species=frames[1].species)
    _equal(srv.wait(tb, timeout_ms=60000), ref[1])
    assert not srv.poll(ta)
    srv.inject("release_held")
    _equal(srv.wait(ta, timeout_ms=60000), ref[0])
    srv.close()


def test_failed_completion_reports_error_and_server_goes_on(ptm, torch):
    from paper_1603_05143_gb300 import PTMError, Server
    frames = _frames()[:2]
    ref = _reference(ptm, torch, frames)
    srv = Server(ptm, streams=2, max_batch_frames=1)
    srv.inject("fail_next")
    ta = srv.submit(frames[0].positions, frames[0].cell, frames[0].pbc, species=frames[0].species)
    with pytest.raises(PTMError) as e:
        srv.wait(ta, timeout_ms=60000)
    assert e.value.status == 3                        # PTM_ERR_CUDA
    tb = srv.submit(frames[1].positions, frames[1].cell, frames[1].pbc, species=frames[1].species)
    _equal(srv.wait(tb, timeout_ms=60000), ref[1])
    srv.close()


def test_destroy_with_held_completion_does_not_hang(ptm, torch):
    from paper_1603_05143_gb300 import Server
    f = _frames()[0]
    srv = Server(ptm, streams=2)
    srv.inject("hold_next")
    srv.submit(f.positions, f.cell, f.pbc, species=f.species)
    srv.close()                                        # drains: the held completion is seen again


def test_resubmit_unfinished_frames_after_destroy_and_create(torch):
    """Frames are stateless: a client that lost its context and server with
    frames outstanding re-submits them to a new context and server and gets
    the same outputs as the frames finished before the loss."""
    from paper_1603_05143_gb300 import PTM, Server
    frames = _frames()
    p1 = PTM(0)
    ref = _reference(p1, torch, frames)
    s1 = Server(p1, streams=2, max_batch_frames=2)
    tickets = [s1.submit(f.positions, f.cell, f.pbc, species=f.species) for f in frames]
    done = {}
    for i in (0, 1):
        done[i] = {k: v.copy() for k, v in s1.wait(tickets[i], timeout_ms=60000).items()}
    s1.close()                                         # the rest are treated as lost
    p1.close()
    p2 = PTM(0)
    s2 = Server(p2, streams=2, max_batch_frames=2)
    again = {i: s2.submit(frames[i].positions, frames[i].cell, frames[i].pbc, species=frames[i].species)
             for i in range(2, len(frames))}
    for i, t in again.items():
        done[i] = s2.wait(t, timeout_ms=60000)
    for i in range(len(frames)):
        _equal(done[i], ref[i])
    s2.close()
    p2.close()
