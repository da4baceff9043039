"""The allocation-free entry point gives the same per-atom results as the
allocating one (GPU only).

ptm_classify_frame_noalloc serves callers that cannot let a library call
cudaMalloc (applications that own all device memory, or in-situ analysis
inside a running simulation).  It keeps its workspace in a static device
array, so this test runs it three times in a row on different frames: a small
float32 frame with atoms outside the cell (which sets the array's wrap and
overshoot words), a larger float64 frame, then a smaller float32 frame with
another cell grid and every atom inside the cell.  Leftovers of one call must
not leak into the next, including beyond the extent of a smaller frame.  The file sorts last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes as C
import math

import numpy as np
import pytest

from paper_1603_05143_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"rmsd": 1e-5, "scale": 1e-5, "quat": 1e-5, "strain": 1e-5}
EXACT = ("structure", "alloy", "correspondence")


def _device_frame(binding, frame, torch):
    pos = torch.from_numpy(np.ascontiguousarray(frame.positions)).cuda()
    sp = None if frame.species is None else torch.from_numpy(frame.species.astype(np.int8)).cuda()
    code = binding.PTM_F64 if frame.positions.dtype == np.float64 else binding.PTM_F32
    f = binding._frame(frame.n, pos.data_ptr(), code, None if sp is None else sp.data_ptr(), frame.cell,
                       frame.pbc, binding.MASK_ALL, math.inf)
    return f, (pos, sp)


def _outputs(binding, n, torch):
    out = binding.allocate_outputs(n, "cuda")
    o = binding.ptm_outputs()
    for name in binding.OUTPUT_NAMES:
        setattr(o, name, out[name].data_ptr())
    return out, o


def test_noalloc_matches_allocating_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_05143_gb300 import binding
    lib = binding.load()
    ptm = binding.PTM(0)
    stream = torch.cuda.current_stream()
    first = I.crystal("l12", I.A_L12, 6, sigma=0.1, seed=3, dtype=np.float64,
                      rotation=I.random_rotation(I.rng_for(1)))
    shift = I.rng_for(2).integers(-1, 2, (first.n, 3)) @ first.cell          # unwrapped positions
    first = I.Frame((first.positions + shift).astype(np.float32), first.cell, first.pbc, first.species, "unwrapped")
    frames = [first,
              I.crystal("bcc", I.A_BCC_FE, 9, sigma=0.15, seed=4, dtype=np.float64),
              I.crystal("fcc", I.A_FCC_CU, (3, 4, 5), sigma=0.05, seed=5, dtype=np.float32,
                        rotation=I.random_rotation(I.rng_for(6)))]
    for frame in frames:                      # three calls in a row, different frames
        f, keep = _device_frame(binding, frame, torch)
        ref = ptm.classify(keep[0], frame.cell, frame.pbc, species=keep[1])
        out, o = _outputs(binding, frame.n, torch)
        rc = lib.ptm_classify_frame_noalloc(C.byref(f), C.byref(o), C.c_void_p(stream.cuda_stream))
        assert rc == 0, binding.STATUS[rc]
        torch.cuda.synchronize()
        for k in EXACT:
            assert torch.equal(out[k], ref[k]), k
        for k, tol in TOL.items():
            a, b = out[k], ref[k]
            fin = torch.isfinite(b)
            assert torch.equal(torch.isfinite(a), fin), k
            assert float((a[fin] - b[fin]).abs().max()) <= tol, k
        assert int((out["structure"] > 0).sum()) > 0.9 * frame.n
    ptm.close()


def test_noalloc_rejects_frames_above_its_limit():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_05143_gb300 import binding
    lib = binding.load()
    frame = I.crystal("fcc", I.A_FCC_CU, 21, sigma=0.05, seed=1, dtype=np.float32)   # 37044 atoms
    f, keep = _device_frame(binding, frame, torch)
    out, o = _outputs(binding, frame.n, torch)
    assert lib.ptm_classify_frame_noalloc(C.byref(f), C.byref(o), None) == 1      # PTM_ERR_INVALID_ARG
