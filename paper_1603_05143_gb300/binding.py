"""ctypes binding of libptm.so: same names as include/ptm.h, marshalling only."""
from __future__ import annotations

import ctypes as C
import math
import pathlib

import numpy as np

_LIB_PATH = pathlib.Path(__file__).resolve().parent / "_build" / "libptm.so"

STRUCTURES = ("NONE", "SC", "FCC", "HCP", "ICO", "BCC")
ALLOYS = ("NONE", "PURE", "L10", "L12_MAJ", "L12_MIN", "B2")
MASK_SC, MASK_FCC, MASK_HCP, MASK_ICO, MASK_BCC, MASK_ALL = 1, 2, 4, 8, 16, 31
PTM_F32, PTM_F64 = 0, 1
STATUS = ("PTM_OK", "PTM_ERR_INVALID_ARG", "PTM_ERR_OUT_OF_MEMORY", "PTM_ERR_CUDA", "PTM_ERR_TIMEOUT",
          "PTM_ERR_DEVICE_STATUS", "PTM_ERR_BUSY", "PTM_ERR_NOT_FOUND")
OUTPUT_NAMES = ("structure", "alloy", "rmsd", "scale", "quat", "strain", "correspondence")
DERIVED_NAMES = ("von_mises", "rodrigues")           # post-processing outputs, on request
OUTPUT_FIELDS = OUTPUT_NAMES + DERIVED_NAMES          # order of ptm_outputs


class ptm_options(C.Structure):
    _fields_ = [("device", C.c_int), ("hbm_budget_bytes", C.c_size_t), ("precision", C.c_int)]


class ptm_frame(C.Structure):
    _fields_ = [("n_atoms", C.c_int64), ("positions", C.c_void_p), ("pos_dtype", C.c_int),
                ("species", C.c_void_p), ("cell", C.c_double * 9), ("pbc", C.c_uint8 * 3),
                ("template_mask", C.c_uint32), ("rmsd_max", C.c_double), ("ordering", C.c_int)]


class ptm_outputs(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in OUTPUT_FIELDS]


class ptm_stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("atoms", "matched", "knn_wide", "knn_fail", "sos", "qcp_fp64",
                                         "tie_fp64", "internal", "candidates", "candidate_points")] + \
               [("pipeline_ms", C.c_double), ("atom_kernel_ms", C.c_double), ("topo_fp64", C.c_int64),
                ("knn_fp64", C.c_int64), ("classify_kernel_ms", C.c_double), ("excluded", C.c_int64),
                ("match_kernel_ms", C.c_double), ("kernel_launches", C.c_int64)]


class ptm_tuning(C.Structure):
    _fields_ = [("cell_factor", C.c_double), ("tile_atoms", C.c_int), ("blocks_per_sm", C.c_int)]


class ptm_server_options(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_batch_frames", C.c_int), ("streams", C.c_int),
                ("tuning", ptm_tuning), ("max_batch_atoms", C.c_int64)]


class PTMError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        name = STATUS[status] if 0 <= status < len(STATUS) else f"status {status}"
        super().__init__(f"{what}: {name}" + (f" ({detail})" if detail else ""))
        self.status = status


_lib = None


def load():
    """Load libptm.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise RuntimeError(f"libptm.so not built ({_LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(str(_LIB_PATH))
        P = C.c_void_p
        L.ptm_create.argtypes = [C.POINTER(ptm_options), C.POINTER(C.c_void_p)]
        L.ptm_destroy.argtypes = [P]
        L.ptm_classify_frame.argtypes = [P, C.POINTER(ptm_frame), C.POINTER(ptm_outputs), P]
        L.ptm_classify_frame_host.argtypes = [P, C.POINTER(ptm_frame), C.POINTER(ptm_outputs), P]
        L.ptm_get_stats.argtypes = [P, C.POINTER(ptm_stats)]
        L.ptm_classify_frame_noalloc.argtypes = [C.POINTER(ptm_frame), C.POINTER(ptm_outputs), P]
        L.ptm_classify_frame_noalloc.restype = C.c_int
        L.ptm_batch_create.argtypes = [P, C.c_int, C.POINTER(ptm_frame), C.POINTER(ptm_outputs),
                                       C.POINTER(ptm_tuning), C.POINTER(C.c_void_p)]
        L.ptm_batch_run.argtypes = [P, P]
        L.ptm_batch_capture.argtypes = [P, P]
        L.ptm_batch_stats.argtypes = [P, C.POINTER(ptm_stats)]
        L.ptm_batch_destroy.argtypes = [P]
        L.ptm_autotune_batch.argtypes = [P, C.c_int, C.POINTER(ptm_frame), C.POINTER(ptm_outputs), P,
                                         C.POINTER(ptm_tuning)]
        for f in ("ptm_batch_create", "ptm_batch_run", "ptm_batch_capture", "ptm_batch_stats",
                  "ptm_batch_destroy", "ptm_autotune_batch"):
            getattr(L, f).restype = C.c_int
        L.ptm_server_create.argtypes = [P, C.POINTER(ptm_server_options), C.POINTER(C.c_void_p)]
        L.ptm_submit.argtypes = [P, C.POINTER(ptm_frame), C.POINTER(ptm_outputs), C.POINTER(C.c_uint64)]
        L.ptm_poll.argtypes = [P, C.c_uint64, C.POINTER(C.c_int)]
        L.ptm_wait.argtypes = [P, C.c_uint64, C.c_int]
        L.ptm_ticket_info.argtypes = [P, C.c_uint64, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        L.ptm_release.argtypes = [P, C.c_uint64]
        L.ptm_server_destroy.argtypes = [P]
        L.ptm_server_inject.argtypes = [P, C.c_int]
        for f in ("ptm_server_create", "ptm_submit", "ptm_poll", "ptm_wait", "ptm_ticket_info", "ptm_release",
                  "ptm_server_destroy", "ptm_server_inject"):
            getattr(L, f).restype = C.c_int
        L.ptm_rmsd_histogram.argtypes = [P, C.c_int64, P, P, C.c_int, C.c_double, P, P]
        L.ptm_rmsd_histogram.restype = C.c_int
        L.ptm_measure_fma_peak.argtypes = [C.c_int, P, C.POINTER(C.c_double)]
        L.ptm_measure_fma_peak.restype = C.c_int
        L.ptm_status_string.argtypes = [C.c_int]
        L.ptm_status_string.restype = C.c_char_p
        L.ptm_last_cuda_error.argtypes = [P]
        L.ptm_last_cuda_error.restype = C.c_char_p
        for f in ("ptm_create", "ptm_destroy", "ptm_classify_frame", "ptm_classify_frame_host", "ptm_get_stats"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def measure_fma_peak(kind="fp32", device=0, stream=None) -> float:
    """Measured FMA throughput (flop/s) of a device (``ptm_measure_fma_peak``):
    kind "fp32" or "fp64"."""
    import torch
    k = {"fp32": 0, "fp64": 1}[kind]
    with torch.cuda.device(device):
        st = stream if stream is not None else torch.cuda.current_stream(device)
        v = C.c_double()
        rc = load().ptm_measure_fma_peak(k, C.c_void_p(st.cuda_stream), C.byref(v))
    if rc:
        raise PTMError(rc, "ptm_measure_fma_peak")
    return v.value


ORDERINGS = {"euclidean": 0, "topological": 1}


def _frame(n, pos_ptr, dtype_code, species_ptr, cell, pbc, mask, rmsd_max, ordering="euclidean") -> ptm_frame:
    f = ptm_frame()
    f.n_atoms = int(n)
    f.positions = pos_ptr
    f.pos_dtype = dtype_code
    f.species = species_ptr
    cell = np.asarray(cell, np.float64).reshape(9)
    for i in range(9):
        f.cell[i] = float(cell[i])
    for i in range(3):
        f.pbc[i] = 1 if pbc[i] else 0
    f.template_mask = int(mask)
    f.rmsd_max = float(rmsd_max) if rmsd_max is not None else math.inf
    f.ordering = ORDERINGS[ordering]
    return f


class PTM:
    """A library context on one CUDA device (``ptm_create`` / ``ptm_destroy``)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, precision: str = "fp32"):
        """precision "fp32" (the product path) or "fp64" (every candidate and the
        winner's outputs in FP64: the one-frame-per-launch comparison form)."""
        self.lib = load()
        opt = ptm_options(device, hbm_budget_bytes, {"fp32": 0, "fp64": 1}[precision])
        h = C.c_void_p()
        rc = self.lib.ptm_create(C.byref(opt), C.byref(h))
        if rc:
            raise PTMError(rc, "ptm_create")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            self.lib.ptm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc:
            raise PTMError(rc, what, self.lib.ptm_last_cuda_error(self.h).decode())

    # ---------------------------------------------------------------- device
    def classify(self, positions, cell, pbc=(True, True, True), species=None, mask=MASK_ALL,
                 rmsd_max=math.inf, out=None, outputs=OUTPUT_NAMES, stream=None, ordering="euclidean"):
        """Classify every atom of a frame held in CUDA tensors (``ptm_classify_frame``).

        positions: (n, 3) float32 or float64 CUDA tensor; species: (n,) int8 or None.
        Returns a dict of CUDA tensors (allocated unless ``out`` provides them);
        the work is enqueued on ``stream`` (default: torch's current stream).
        """
        import torch
        if not positions.is_cuda or positions.dim() != 2 or positions.shape[1] != 3:
            raise ValueError("positions must be an (n, 3) CUDA tensor")
        positions = positions.contiguous()
        n = positions.shape[0]
        dev = positions.device
        if positions.dtype == torch.float32:
            code = PTM_F32
        elif positions.dtype == torch.float64:
            code = PTM_F64
        else:
            raise ValueError("positions must be float32 or float64")
        sp_ptr = None
        if species is not None:
            species = species.to(device=dev, dtype=torch.int8).contiguous()
            sp_ptr = species.data_ptr()
        if out is None:
            out = allocate_outputs(n, dev, outputs)
        o = ptm_outputs()
        for name in OUTPUT_FIELDS:
            t = out.get(name)
            setattr(o, name, t.data_ptr() if t is not None else None)
        f = _frame(n, positions.data_ptr(), code, sp_ptr, cell, pbc, mask, rmsd_max, ordering)
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        self._keep = (positions, species)
        self._check(self.lib.ptm_classify_frame(self.h, C.byref(f), C.byref(o), C.c_void_p(st.cuda_stream)),
                    "ptm_classify_frame")
        return out

    # ------------------------------------------------------------------ host
    def classify_host(self, positions, cell, pbc=(True, True, True), species=None, mask=MASK_ALL,
                      rmsd_max=math.inf, out=None, outputs=OUTPUT_NAMES, stream=None, ordering="euclidean"):
        """Same as ``classify`` for host (numpy) buffers (``ptm_classify_frame_host``):
        the library copies to and from the device and returns when done."""
        pos = np.ascontiguousarray(positions)
        if pos.dtype not in (np.float32, np.float64) or pos.ndim != 2 or pos.shape[1] != 3:
            raise ValueError("positions must be an (n, 3) float32/float64 array")
        n = pos.shape[0]
        sp = None if species is None else np.ascontiguousarray(species, np.int8)
        if out is None:
            out = allocate_outputs_host(n, outputs)
        o = ptm_outputs()
        for name in OUTPUT_FIELDS:
            a = out.get(name)
            setattr(o, name, a.ctypes.data if a is not None else None)
        f = _frame(n, pos.ctypes.data, PTM_F64 if pos.dtype == np.float64 else PTM_F32,
                   sp.ctypes.data if sp is not None else None, cell, pbc, mask, rmsd_max, ordering)
        st = 0 if stream is None else stream.cuda_stream
        self._check(self.lib.ptm_classify_frame_host(self.h, C.byref(f), C.byref(o), C.c_void_p(st)),
                    "ptm_classify_frame_host")
        return out

    def rmsd_histogram(self, structure, rmsd, nbins=100, rmsd_max=0.5, stream=None):
        """Per-structure RMSD histogram (``ptm_rmsd_histogram``) of outputs held in
        CUDA tensors: int64 tensor (5, nbins + 1), rows SC..BCC, last column =
        at or beyond rmsd_max."""
        import torch
        n = int(structure.shape[0])
        if rmsd.shape[0] != n or not (structure.is_cuda and rmsd.is_cuda):
            raise ValueError("structure and rmsd must be CUDA tensors of the same length")
        structure = structure.contiguous()
        rmsd = rmsd.contiguous()
        counts = torch.empty((5, nbins + 1), dtype=torch.int64, device=structure.device)
        st = stream if stream is not None else torch.cuda.current_stream(structure.device)
        self._check(self.lib.ptm_rmsd_histogram(self.h, n, C.c_void_p(structure.data_ptr()),
                                                C.c_void_p(rmsd.data_ptr()), int(nbins), float(rmsd_max),
                                                C.c_void_p(counts.data_ptr()), C.c_void_p(st.cuda_stream)),
                    "ptm_rmsd_histogram")
        return counts

    def stats(self) -> dict:
        s = ptm_stats()
        self._check(self.lib.ptm_get_stats(self.h, C.byref(s)), "ptm_get_stats")
        return {k: getattr(s, k) for k, _ in ptm_stats._fields_}

    # --------------------------------------------------------------- batches
    def batch(self, frames, mask=MASK_ALL, rmsd_max=math.inf, tuning=None, outputs=OUTPUT_NAMES):
        """A ``Batch`` over frames given as dicts with CUDA tensors
        ``positions`` (n, 3), optional ``species`` (n,), and ``cell``, ``pbc``."""
        return Batch(self, frames, mask, rmsd_max, tuning, outputs)

    def autotune(self, frames, mask=MASK_ALL, rmsd_max=math.inf, stream=None, cache=None):
        """Fastest ptm_tuning for these frames (``ptm_autotune_batch``), cached in a
        JSON file keyed by device name and workload signature."""
        import json
        import os
        import torch
        key = None
        if cache:
            name = torch.cuda.get_device_name(self.device)
            n = [int(f["positions"].shape[0]) for f in frames]
            key = f"{name}|{len(n)}|{sum(n)}|{min(n)}|{max(n)}|{frames[0]['positions'].dtype}"
            if os.path.exists(cache):
                data = json.load(open(cache))
                if key in data:
                    return data[key]
        fr, outs, keep, _ = _batch_structs(frames, mask, rmsd_max, OUTPUT_NAMES)
        best = ptm_tuning()
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._check(self.lib.ptm_autotune_batch(self.h, len(frames), fr, outs, C.c_void_p(st.cuda_stream),
                                                C.byref(best)), "ptm_autotune_batch")
        res = {"cell_factor": best.cell_factor, "tile_atoms": best.tile_atoms, "blocks_per_sm": best.blocks_per_sm}
        if cache:
            data = json.load(open(cache)) if os.path.exists(cache) else {}
            data[key] = res
            os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
            json.dump(data, open(cache, "w"), indent=1)
        return res


def _batch_structs(frames, mask, rmsd_max, outputs):
    import torch
    n = len(frames)
    fr = (ptm_frame * n)()
    outs = (ptm_outputs * n)()
    keep, out_tensors = [], []
    for i, f in enumerate(frames):
        pos = f["positions"].contiguous()
        sp = f.get("species")
        if sp is not None:
            sp = sp.to(device=pos.device, dtype=torch.int8).contiguous()
        code = PTM_F64 if pos.dtype == torch.float64 else PTM_F32
        fr[i] = _frame(pos.shape[0], pos.data_ptr(), code, None if sp is None else sp.data_ptr(), f["cell"],
                       f.get("pbc", (True, True, True)), mask, rmsd_max, f.get("ordering", "euclidean"))
        o = allocate_outputs(pos.shape[0], pos.device, outputs)
        for name in OUTPUT_FIELDS:
            t = o.get(name)
            setattr(outs[i], name, t.data_ptr() if t is not None else None)
        keep.append((pos, sp))
        out_tensors.append(o)
    return fr, outs, keep, out_tensors


class Batch:
    """Frames classified together by one persistent launch (``ptm_batch_*``)."""

    def __init__(self, ptm, frames, mask=MASK_ALL, rmsd_max=math.inf, tuning=None, outputs=OUTPUT_NAMES):
        self.ptm = ptm
        self.lib = ptm.lib
        fr, outs, self._keep, self.outputs = _batch_structs(frames, mask, rmsd_max, outputs)
        t = None
        if tuning:
            t = ptm_tuning(float(tuning.get("cell_factor", 0)), int(tuning.get("tile_atoms", 0)),
                           int(tuning.get("blocks_per_sm", 0)))
        h = C.c_void_p()
        ptm._check(self.lib.ptm_batch_create(ptm.h, len(frames), fr, outs, C.byref(t) if t else None, C.byref(h)),
                   "ptm_batch_create")
        self.h = h
        self._structs = (fr, outs)

    def _stream(self, stream):
        import torch
        return stream if stream is not None else torch.cuda.current_stream(self.ptm.device)

    def run(self, stream=None):
        self.ptm._check(self.lib.ptm_batch_run(self.h, C.c_void_p(self._stream(stream).cuda_stream)), "ptm_batch_run")

    def capture(self, stream):
        self.ptm._check(self.lib.ptm_batch_capture(self.h, C.c_void_p(stream.cuda_stream)), "ptm_batch_capture")

    def stats(self) -> dict:
        s = ptm_stats()
        self.ptm._check(self.lib.ptm_batch_stats(self.h, C.byref(s)), "ptm_batch_stats")
        return {k: getattr(s, k) for k, _ in ptm_stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.ptm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def allocate_outputs(n, device, outputs=OUTPUT_NAMES):
    import torch
    shapes = {"structure": ((n,), torch.int8), "alloy": ((n,), torch.int8), "rmsd": ((n,), torch.float32),
              "scale": ((n,), torch.float32), "quat": ((n, 4), torch.float32),
              "strain": ((n, 3, 3), torch.float32), "correspondence": ((n, 15), torch.int32),
              "von_mises": ((n,), torch.float32), "rodrigues": ((n, 3), torch.float32)}
    return {k: torch.empty(*shapes[k][0], dtype=shapes[k][1], device=device) for k in outputs}


def allocate_outputs_host(n, outputs=OUTPUT_NAMES, pinned=False):
    shapes = {"structure": ((n,), np.int8), "alloy": ((n,), np.int8), "rmsd": ((n,), np.float32),
              "scale": ((n,), np.float32), "quat": ((n, 4), np.float32), "strain": ((n, 3, 3), np.float32),
              "correspondence": ((n, 15), np.int32), "von_mises": ((n,), np.float32),
              "rodrigues": ((n, 3), np.float32)}
    if pinned:
        import torch
        tt = {np.int8: torch.int8, np.float32: torch.float32, np.int32: torch.int32}
        return {k: torch.empty(shapes[k][0], dtype=tt[shapes[k][1]], pin_memory=True).numpy() for k in outputs}
    return {k: np.empty(shapes[k][0], shapes[k][1]) for k in outputs}


class Server:
    """Continuous-batching server (``ptm_server_*``) for frames held in host memory.

    ``submit`` returns a ticket immediately; the frame's outputs (numpy arrays,
    page-locked when ``pinned``) are filled when the ticket completes."""

    def __init__(self, ptm, hbm_budget_bytes=0, max_batch_frames=0, streams=0, tuning=None, max_batch_atoms=0):
        self.ptm = ptm
        self.lib = ptm.lib
        t = tuning or {}
        opt = ptm_server_options(int(hbm_budget_bytes), int(max_batch_frames), int(streams),
                                 ptm_tuning(float(t.get("cell_factor", 0)), int(t.get("tile_atoms", 0)),
                                            int(t.get("blocks_per_sm", 0))), int(max_batch_atoms))
        h = C.c_void_p()
        ptm._check(self.lib.ptm_server_create(ptm.h, C.byref(opt), C.byref(h)), "ptm_server_create")
        self.h = h
        self._live = {}

    def submit(self, positions, cell, pbc=(True, True, True), species=None, mask=MASK_ALL, rmsd_max=math.inf,
               out=None, pinned=False, ordering="euclidean"):
        pos = np.ascontiguousarray(positions)
        n = pos.shape[0]
        sp = None if species is None else np.ascontiguousarray(species, np.int8)
        if out is None:
            out = allocate_outputs_host(n, pinned=pinned)
        o = ptm_outputs()
        for name in OUTPUT_FIELDS:
            a = out.get(name)
            setattr(o, name, a.ctypes.data if a is not None else None)
        f = _frame(n, pos.ctypes.data, PTM_F64 if pos.dtype == np.float64 else PTM_F32,
                   sp.ctypes.data if sp is not None else None, cell, pbc, mask, rmsd_max, ordering)
        t = C.c_uint64()
        rc = self.lib.ptm_submit(self.h, C.byref(f), C.byref(o), C.byref(t))
        if rc:
            raise PTMError(rc, "ptm_submit")
        self._live[t.value] = (pos, sp, out)          # keep the host buffers alive
        return t.value

    def poll(self, ticket) -> bool:
        d = C.c_int()
        rc = self.lib.ptm_poll(self.h, ticket, C.byref(d))
        if rc:
            raise PTMError(rc, "ptm_poll")
        return bool(d.value)

    def wait(self, ticket, timeout_ms=-1):
        """Outputs of the ticket; raises PTMError (PTM_ERR_TIMEOUT, ...) otherwise."""
        rc = self.lib.ptm_wait(self.h, ticket, int(timeout_ms))
        if rc:
            raise PTMError(rc, "ptm_wait")
        return self._live[ticket][2]

    def info(self, ticket):
        times = (C.c_double * 3)()
        b = C.c_int64()
        rc = self.lib.ptm_ticket_info(self.h, ticket, times, C.byref(b))
        if rc:
            raise PTMError(rc, "ptm_ticket_info")
        return {"submit": times[0], "start": times[1], "done": times[2], "batch": b.value}

    def release(self, ticket):
        self.lib.ptm_release(self.h, ticket)
        self._live.pop(ticket, None)

    FAULTS = {"hold_next": 1, "release_held": 2, "fail_next": 3}

    def inject(self, fault: str):
        """Host-side fault injection (``ptm_server_inject``): "hold_next",
        "release_held" or "fail_next"."""
        rc = self.lib.ptm_server_inject(self.h, self.FAULTS[fault])
        if rc:
            raise PTMError(rc, "ptm_server_inject")

    def close(self):
        if getattr(self, "h", None):
            self.lib.ptm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
