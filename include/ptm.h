/*
 * ptm.h -- C ABI of the GB300 per-atom Polyhedral Template Matching library
 * (libptm.so).  Method: Larsen, Schmidt & Schiotz, "Robust Structural
 * Identification via Polyhedral Template Matching".
 *
 * For every atom of a periodic frame the library
 *   - selects the 14 nearest neighbours, Euclidean order (Sec. 3, Table 1);
 *   - builds the convex hulls of the first 6, 12 and 14 neighbours and labels
 *     each hull graph by a Weinberg walk, looked up among the codes of the
 *     template triangulations (Sec. 4);
 *   - matches the labels against the SC, FCC, HCP, ICO and BCC templates and
 *     evaluates the scale-invariant RMSD (Eq. 3-4) of every admissible
 *     correspondence (Algorithm 1);
 *   - returns structure type, RMSD, scale, orientation (Sec. 7), elastic strain
 *     (Sec. 8, Eq. 6-7) and the binary alloy label (Sec. 6, Table 3).
 *
 * All compute runs in CUDA kernels on the device chosen at ptm_create.
 * No function aborts or throws across this boundary: every failure is a
 * ptm_status.  Functions are not thread-safe on one context; use one context
 * per host thread.
 */
#ifndef PTM_H
#define PTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ptm_context ptm_context;   /* opaque, owned by the library */

typedef enum {
  PTM_OK = 0,
  PTM_ERR_INVALID_ARG = 1,     /* a NULL pointer, bad size, singular cell, unknown dtype */
  PTM_ERR_OUT_OF_MEMORY = 2,   /* device workspace could not be allocated */
  PTM_ERR_CUDA = 3,            /* a CUDA runtime call failed; see ptm_last_cuda_error */
  PTM_ERR_TIMEOUT = 4,         /* a bounded wait ran out (serving) */
  PTM_ERR_DEVICE_STATUS = 5,   /* a kernel reported an internal inconsistency */
  PTM_ERR_BUSY = 6,            /* no serving slot or memory budget free right now */
  PTM_ERR_NOT_FOUND = 7        /* unknown serving ticket */
} ptm_status;

/* Template mask bits, in the order Algorithm 1 visits the templates. */
enum { PTM_MASK_SC = 1, PTM_MASK_FCC = 2, PTM_MASK_HCP = 4, PTM_MASK_ICO = 8,
       PTM_MASK_BCC = 16, PTM_MASK_ALL = 31 };

/* Structure codes written to ptm_outputs.structure. */
enum { PTM_NONE = 0, PTM_SC = 1, PTM_FCC = 2, PTM_HCP = 3, PTM_ICO = 4, PTM_BCC = 5 };

/* Binary alloy labels (Sec. 6): FCC uses the coplanar groups of Table 3, BCC the
   two neighbour shells.  "same"/"other" are relative to the central atom. */
enum { PTM_ALLOY_NONE = 0, PTM_ALLOY_PURE = 1, PTM_ALLOY_L10 = 2, PTM_ALLOY_L12_MAJ = 3,
       PTM_ALLOY_L12_MIN = 4, PTM_ALLOY_B2 = 5 };

/* Position element types. */
enum { PTM_F32 = 0, PTM_F64 = 1 };

/* Neighbour ordering (Sec. 3, Eq. 5).  Euclidean: the 14 nearest images by
   distance (then atom id, then image), distances compared in FP64 whatever the
   position type (float32 positions are widened exactly; the library decides in
   FP32 wherever a proven FP32 error bound separates two distances).  Topological: the 18 nearest, reordered
   by the area of the face their Voronoi cell shares with the atom's (the cell
   taken among those 18), larger first, then nearer; areas within 1e-3 of the
   mean squared neighbour distance count as equal; the first 14 are used.
   Topological ordering adds one per-atom kernel (about the cost of the rest). */
enum { PTM_ORDER_EUCLIDEAN = 0, PTM_ORDER_TOPOLOGICAL = 1 };

/* Arithmetic of the metric steps (QCP, selection, outputs).  The exact hull
   predicates, Weinberg codes and lookup are the same in both. */
enum {
  PTM_PREC_FP32 = 0,         /* FP32, with FP64 where stability needs it (the product path) */
  PTM_PREC_FP64 = 1          /* every candidate and the winner's outputs in FP64: the
                                one-frame-per-launch comparison form; ptm_classify_frame
                                and ptm_classify_frame_host only (batches and servers
                                always use PTM_PREC_FP32) */
};

typedef struct {
  int device;                /* CUDA device ordinal */
  size_t hbm_budget_bytes;   /* serving admission budget; 0 = half the free memory at create */
  int precision;             /* PTM_PREC_FP32 (0) or PTM_PREC_FP64 */
} ptm_options;

/* One frame.  Problem statement of Algorithm 1: positions of every atom, the
   periodic cell, optional species (Sec. 6), the template set and RMSD_max
   (Sec. 5.1). */
typedef struct {
  int64_t n_atoms;           /* >= 1 and < 2^31 */
  const void *positions;     /* n_atoms x 3, row-major, element type pos_dtype */
  int pos_dtype;             /* PTM_F32 or PTM_F64 */
  const int8_t *species;     /* n_atoms species codes, or NULL (alloy = NONE) */
  double cell[9];            /* row-major; rows are the three cell vectors (Angstrom) */
  uint8_t pbc[3];            /* 1 = periodic along cell vector i */
  uint32_t template_mask;    /* PTM_MASK_* bits; 0 means PTM_MASK_ALL */
  double rmsd_max;           /* atoms whose best RMSD exceeds it are unmatched; INFINITY = none */
  int ordering;              /* neighbour ordering (Sec. 3): PTM_ORDER_EUCLIDEAN (0) or
                                PTM_ORDER_TOPOLOGICAL (not by ptm_classify_frame_noalloc) */
} ptm_frame;

/* Per-atom outputs, indexed by atom.  Any pointer may be NULL to skip it.
   Unmatched atoms (Algorithm 1: r* = infinity, structure disordered) get
   structure PTM_NONE, rmsd +INF, scale 0, quat (1,0,0,0), strain 0,
   correspondence -1, alloy PTM_ALLOY_NONE, von_mises 0, rodrigues 0. */
typedef struct {
  int8_t *structure;         /* n: PTM_NONE .. PTM_BCC */
  int8_t *alloy;             /* n: PTM_ALLOY_* */
  float *rmsd;               /* n: scale-invariant RMSD of the best match, Eq. 3 */
  float *scale;              /* n: the optimal s of Eq. 3 (data -> template units) */
  float *quat;               /* n x 4: (w, x, y, z), w >= 0: rotation taking the template
                                onto the neighbourhood, reduced to the fundamental zone */
  float *strain;             /* n x 9: symmetric P of the left polar decomposition A = P U
                                of the least-squares deformation gradient (Eq. 6-7) */
  int32_t *correspondence;   /* n x 15: atom index mapped to template slot 0..k
                                (slot 0 = the atom itself), -1 beyond k; the smallest
                                member of its orbit under the template symmetry */
  /* derived outputs (post-processing, written only when requested) */
  float *von_mises;          /* n: von Mises shear strain of P (Sec. 8),
                                sqrt(3/2 sum P_ij^2 - 1/2 (tr P)^2); 0 when unmatched */
  float *rodrigues;          /* n x 3: Rodrigues-Frank vector (x, y, z) / w of quat
                                (Sec. 7); 0 when unmatched */
} ptm_outputs;

/* Counters of the last completed classify call (rates of the rare paths). */
typedef struct {
  int64_t atoms;             /* atoms processed */
  int64_t matched;           /* atoms with a structure */
  int64_t knn_wide;          /* atoms whose neighbour search needed more than 27 cells */
  int64_t knn_fail;          /* atoms whose search gave up (left unmatched) */
  int64_t sos;               /* orientation tests decided by Simulation of Simplicity */
  int64_t qcp_fp64;          /* candidates re-solved in FP64: small eigenvalue gap */
  int64_t tie_fp64;          /* atoms whose best candidates were re-ranked in FP64 */
  int64_t internal;          /* internal inconsistencies (should be 0) */
  int64_t candidates;        /* correspondences scored by QCP (symmetry-reduced, Appendix A) */
  int64_t candidate_points;  /* sum over those correspondences of the point count N = k + 1 */
  double pipeline_ms;        /* device time of the whole call (cell list + classification) */
  double atom_kernel_ms;     /* device time of the per-atom kernels (neighbour lists +
                                classification) */
  int64_t topo_fp64;         /* atoms whose topological order was decided in FP64 (an area
                                gap at the edge of the equal-area band) */
  int64_t knn_fp64;          /* float32 input: atoms whose neighbour order needed FP64
                                distances (two candidates within the FP32 error bound) */
  double classify_kernel_ms; /* device time of the classification kernels (hulls, codes,
                                QCP, outputs), after the neighbour lists */
  int64_t excluded;          /* atoms with a non-finite coordinate or more than 100 cell periods
                                outside the cell: left unmatched and nobody's neighbour */
  double match_kernel_ms;    /* device time of the matching kernels alone (QCP, selection,
                                outputs): the last part of classify_kernel_ms */
  int64_t kernel_launches;   /* CUDA kernels the call launched */
} ptm_stats;

/* Create a context on options->device (NULL options: device 0, default budget).
   The context owns all device workspace and frees it in ptm_destroy. */
ptm_status ptm_create(const ptm_options *options, ptm_context **out);

/* Release the context and its workspace.  Waits for its work to finish. */
ptm_status ptm_destroy(ptm_context *ctx);

/* Classify every atom of one frame.  frame->positions, frame->species and all
   output pointers are DEVICE pointers; the call only enqueues work on `stream`
   (a cudaStream_t, NULL = legacy default stream) and returns.  Buffers must stay
   alive until the stream reaches this point.  The first call for a larger frame
   grows the context workspace (cudaMalloc), so warm up before timing or
   capturing.  Errors in the arguments are returned before anything is
   enqueued. */
ptm_status ptm_classify_frame(ptm_context *ctx, const ptm_frame *frame, const ptm_outputs *out,
                              void *stream);

/* Same, but positions, species and outputs are HOST pointers (page-locked memory
   is faster).  The library copies inputs to its own device buffers, classifies,
   copies the outputs back and synchronises `stream` before returning. */
ptm_status ptm_classify_frame_host(ptm_context *ctx, const ptm_frame *frame,
                                   const ptm_outputs *out, void *stream);

/* Copy the counters and device timings of the last classify call (synchronises
   its stream).  Timings come from CUDA events recorded on that stream. */
ptm_status ptm_get_stats(ptm_context *ctx, ptm_stats *out);

/* ---------------------------------------------------------------- batches
   Many frames of uneven size classified by one persistent launch: every frame
   gets its own cell list, one scan covers all cells, and the per-atom kernel
   pulls tiles of atoms from one global queue until the batch is exhausted, so
   small and large frames balance across the GPU.  A batch remembers the
   caller's device buffers; running it again re-reads them (update positions in
   place for the next MD frame of the same size and cell shape). */
typedef struct ptm_batch ptm_batch;

/* Tunables of a batch; a field <= 0 keeps its default.
   cell_factor: cell width / expected 14-neighbour radius (default 1.25);
   tile_atoms: atoms one warp takes from the queue per grab, rounded up to a
   multiple of 32 (default 32, one per lane: each warp grabs on its own, so
   no warp waits for another; larger grabs lengthen the tail when the queue
   runs dry, 64 measured 10 % slower on a 2^20-atom frame);
   blocks_per_sm: resident 64-thread blocks per SM for the persistent grid
   (default 7, the shared-memory limit).  Atoms per warp are fixed at 32 (one
   atom per lane). */
typedef struct {
  double cell_factor;
  int tile_atoms;
  int blocks_per_sm;
} ptm_tuning;

/* Build a batch of n_frames frames (all PTM_F32 or all PTM_F64; device
   buffers; outs[i] belongs to frames[i]).  Allocates the batch workspace
   (about 40 B per atom plus 8 B per cell) and copies the frame descriptors to
   the device.  tuning may be NULL. */
ptm_status ptm_batch_create(ptm_context *ctx, int n_frames, const ptm_frame *frames,
                            const ptm_outputs *outs, const ptm_tuning *tuning, ptm_batch **out);

/* Enqueue the whole batch on `stream`; if the batch was captured, replay its
   CUDA graph instead.  Asynchronous. */
ptm_status ptm_batch_run(ptm_batch *batch, void *stream);

/* Capture one run of the batch into a CUDA graph owned by the batch (stream
   must be a non-NULL capturable stream); later ptm_batch_run calls launch the
   graph. */
ptm_status ptm_batch_capture(ptm_batch *batch, void *stream);

/* Counters and device timings of the batch's last run (waits for it). */
ptm_status ptm_batch_stats(ptm_batch *batch, ptm_stats *out);

/* Free the batch and its workspace (waits for its last run). */
ptm_status ptm_batch_destroy(ptm_batch *batch);

/* Time every candidate tuning on this batch (cell_factor in {1.125, 1.25,
   1.4}, tile_atoms in {32, 64}, blocks_per_sm in {7, 8}) and return the
   fastest in *best.  Runs the batch (every m-th frame of it when it holds more
   than about 40 M atoms) 36 times; outputs are written with the same results
   each time. */
ptm_status ptm_autotune_batch(ptm_context *ctx, int n_frames, const ptm_frame *frames,
                              const ptm_outputs *outs, void *stream, ptm_tuning *best);

/* ---------------------------------------------------------------- serving
   In-situ analysis of MD frames that arrive at any time.  A server owns one
   scheduler thread and a few non-blocking streams.  Submitted frames (HOST
   buffers, ideally page-locked) wait in a FIFO and are admitted when their
   device bytes (inputs, outputs and workspace, about 300 B per atom) fit the
   HBM budget next to the frames already on the device.  Whenever a stream is
   free, the admitted frames not yet launched (up to max_batch_frames and
   max_batch_atoms, in arrival order) form one batch: copy in, one persistent launch, copy out.  Frames arriving while
   batches run join the next batch as memory and streams free up, and batches
   on different streams overlap on the device (continuous batching).  Device
   memory is pooled and reused; nothing is freed while the server runs.  Each
   frame's results equal those of ptm_classify_frame. */
typedef struct ptm_server ptm_server;

typedef struct {
  size_t hbm_budget_bytes;   /* 0 = the context's budget (half the free memory at create) */
  int max_batch_frames;      /* frames per launch; 0 = 64 */
  int streams;               /* batches in flight; 0 = 4, at most 8 */
  ptm_tuning tuning;         /* zeros = defaults */
  int64_t max_batch_atoms;   /* atoms per launch (a larger single frame runs alone);
                                0 = 4,194,304 */
} ptm_server_options;

ptm_status ptm_server_create(ptm_context *ctx, const ptm_server_options *options, ptm_server **out);

/* Queue one frame (HOST pointers; they must stay valid until the ticket
   completes).  Never blocks on the GPU. */
ptm_status ptm_submit(ptm_server *server, const ptm_frame *frame, const ptm_outputs *out,
                      uint64_t *ticket);

/* *done = 1 once the ticket finished (its outputs are on the host); returns the
   frame's status when done (PTM_ERR_OUT_OF_MEMORY if it can never fit the
   budget), PTM_ERR_NOT_FOUND for an unknown ticket. */
ptm_status ptm_poll(ptm_server *server, uint64_t ticket, int *done);

/* Wait at most timeout_ms (< 0: no limit) for a ticket; PTM_ERR_TIMEOUT if it
   is still running, else the frame's status. */
ptm_status ptm_wait(ptm_server *server, uint64_t ticket, int timeout_ms);

/* times[0..2] = submit, launch and completion times (seconds, steady clock);
   *batch = index of the batch that carried the frame (-1 before launch). */
ptm_status ptm_ticket_info(ptm_server *server, uint64_t ticket, double *times, int64_t *batch);

/* Forget a finished ticket (PTM_ERR_BUSY while it runs). */
ptm_status ptm_release(ptm_server *server, uint64_t ticket);

/* Finish all queued and running frames, then free the server. */
ptm_status ptm_server_destroy(ptm_server *server);

/* Host-side fault injection for tests of the serving path (the paper has no
   counterpart; no GPU fault is involved).  PTM_FAULT_HOLD_NEXT: the scheduler
   does not see the completion of the next batch it launches (a lost
   completion) until PTM_FAULT_RELEASE_HELD or ptm_server_destroy; waits on its
   tickets run into their timeouts while other batches complete.
   PTM_FAULT_FAIL_NEXT: the next batch launched completes with PTM_ERR_CUDA, as
   when its completion event reports an error (the server then keeps serving).
   PTM_ERR_INVALID_ARG for another code. */
enum { PTM_FAULT_HOLD_NEXT = 1, PTM_FAULT_RELEASE_HELD = 2, PTM_FAULT_FAIL_NEXT = 3 };
ptm_status ptm_server_inject(ptm_server *server, int fault);

/* Largest frame accepted by ptm_classify_frame_noalloc. */
#define PTM_NOALLOC_MAX_ATOMS 32768

/* Classify one frame of at most PTM_NOALLOC_MAX_ATOMS atoms without allocating
   any memory (the paper has no counterpart: this is a service to callers).
   It is for callers that cannot let a library call cudaMalloc: host
   applications that own all device memory through their own pool, and in-situ
   analysis inside a running simulation, where cudaMalloc and cudaFree may
   synchronise the device and stall the caller's pipeline.  No context is
   needed: the call runs on the current device, on `stream`, with the same
   kernels and results as ptm_classify_frame; positions, species and outputs are
   DEVICE pointers owned by the caller.  Its workspace is one static device
   array of about 7.0 MiB that every GPU loading this library holds until the
   process exits.  Its device address belongs to the CUDA context current at
   the call: every call outside stream capture looks it up again (so a device
   reset or a caller-made driver context is followed), and a call on a
   capturing stream reuses the address last found for the current context, so
   make at least one call outside capture in that context first (else
   PTM_ERR_INVALID_ARG).  All calls share
   the array and keep its last contents (the call clears what must start at
   zero), so calls whose work overlaps on the GPU race: order them on one
   stream.  Returns PTM_ERR_INVALID_ARG for frames above the limit (or bad
   arguments) before enqueueing anything, PTM_ERR_CUDA if a launch fails. */
ptm_status ptm_classify_frame_noalloc(const ptm_frame *frame, const ptm_outputs *out, void *stream);

/* Largest bin count of ptm_rmsd_histogram. */
#define PTM_HIST_MAX_BINS 2048

/* Per-structure histogram of the RMSD of matched atoms (Sec. 5.1: the
   histogram from which RMSD_max is chosen after the analysis), computed on the
   device from outputs of a classify call.  structure, rmsd: DEVICE arrays of
   n_atoms.  counts: DEVICE int64 array of 5 x (nbins + 1), overwritten: row
   S - 1 counts structure S (PTM_SC .. PTM_BCC); column b < nbins counts atoms
   with b <= rmsd * s < b + 1, where s = nbins / rmsd_max rounded to float32 and
   the product is one float32 multiplication; column nbins counts atoms at or
   beyond rmsd_max.  Unmatched atoms (structure PTM_NONE or infinite rmsd) are
   not counted.  Asynchronous on `stream`.  PTM_ERR_INVALID_ARG for NULL
   pointers, n_atoms < 0, nbins outside [1, PTM_HIST_MAX_BINS] or rmsd_max not
   finite and positive. */
ptm_status ptm_rmsd_histogram(ptm_context *ctx, int64_t n_atoms, const int8_t *structure, const float *rmsd,
                              int nbins, double rmsd_max, int64_t *counts, void *stream);

/* Measured FMA throughput of the current device, for the ALU roofline of the
   per-atom kernel (the paper has no counterpart).  kind 0 = FP32, 1 = FP64.
   Launches a kernel of independent FMA chains that fills every SM, on
   `stream` (NULL = legacy default stream), times about 50 ms of it with CUDA
   events (best of three) and stores flop/s (two per FMA) in *flops_per_s.
   Allocates and frees a small device buffer; synchronises `stream`.
   PTM_ERR_INVALID_ARG for another kind or a NULL result pointer,
   PTM_ERR_CUDA if no device is usable. */
ptm_status ptm_measure_fma_peak(int kind, void *stream, double *flops_per_s);

/* Human-readable name of a status; never NULL. */
const char *ptm_status_string(ptm_status status);

/* Message of the last CUDA error seen by this context ("" if none). */
const char *ptm_last_cuda_error(ptm_context *ctx);

#ifdef __cplusplus
}
#endif
#endif /* PTM_H */
