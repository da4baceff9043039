// libptm.so host side: the C ABI of include/ptm.h (Larsen, Schmidt & Schiotz,
// "Robust Structural Identification via Polyhedral Template Matching").
// Validates arguments, sizes the cell list, owns the device workspace and
// enqueues the kernels of ptm_kernels.cuh on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#define PTM_TBL_CONST __constant__ const
#define PTM_TBL_GLOBAL __device__ const
#define PTM_TBL_ALIGN16 __attribute__((aligned(16)))
#include "ptm_kernels.cuh"
#include "ptm_topo.cuh"

// =================================================================== host
using namespace ptm;

struct ptm_context {
  int device = 0;
  int precision = PTM_PREC_FP32;
  size_t budget = 0;
  std::string last_error;
  // workspace
  size_t cap_atoms = 0, cap_cells = 0, cap_sorted_bytes = 0;
  void *sorted = nullptr;
  int *sbin = nullptr, *wrapv = nullptr, *atom_cell = nullptr, *atom_rank = nullptr, *atom_wrap = nullptr;
  int *cell_count = nullptr, *cell_start = nullptr, *block_sums = nullptr;
  int *dstat = nullptr;
  unsigned long long *counters = nullptr;
  ShiftTables *tab = nullptr;      // the current frame's image shifts
  int launches = 0;                // kernels the last call launched
  cudaStream_t last_stream = nullptr;
  cudaEvent_t ev[5] = {};   // call start, per-atom kernels start, end, k_hulls start, k_match start
  // host-buffer entry point
  size_t cap_host_atoms = 0;
  void *hpos = nullptr;
  int8_t *hspecies = nullptr;
  int8_t *o_struct = nullptr, *o_alloy = nullptr;
  float *o_rmsd = nullptr, *o_scale = nullptr, *o_quat = nullptr, *o_strain = nullptr;
  int32_t *o_corr = nullptr;
  float *o_vm = nullptr, *o_rf = nullptr;
  // every atom's 14 neighbours (k_knn or k_topo -> k_hulls, k_match) and its
  // matched snapshots (k_hulls -> k_match)
  int2 *nbr = nullptr;
  uint64_t *lam = nullptr;
  uint32_t *ents = nullptr;
  size_t cap_nbr = 0;
  // topological order: atoms for the FP64 pass ([n] = their count) and what
  // the FP32 pass keeps for it
  int *topo_list = nullptr;
  TopoSide *topo_side = nullptr;
  size_t cap_topo = 0;
};

static ptm_status cuda_fail(ptm_context *ctx, cudaError_t e, const char *what) {
  if (ctx) ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? PTM_ERR_OUT_OF_MEMORY : PTM_ERR_CUDA;
}

#define CK(call)                                                     \
  do {                                                               \
    cudaError_t e_ = (call);                                         \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);         \
  } while (0)

static ptm_status grow(ptm_context *ctx, size_t n, size_t ncell, int f64) {
  size_t sb = n * (f64 ? sizeof(Atom64) : sizeof(float4));
  if (n > ctx->cap_atoms || sb > ctx->cap_sorted_bytes) {
    cudaFree(ctx->sorted); cudaFree(ctx->sbin); cudaFree(ctx->wrapv);
    cudaFree(ctx->atom_cell); cudaFree(ctx->atom_rank); cudaFree(ctx->atom_wrap);
    ctx->sorted = nullptr; ctx->sbin = ctx->wrapv = ctx->atom_cell = ctx->atom_rank = ctx->atom_wrap = nullptr;
    ctx->cap_atoms = ctx->cap_sorted_bytes = 0;
    size_t na = std::max(n, ctx->cap_atoms);
    size_t nsb = std::max(sb, na * (f64 ? sizeof(Atom64) : sizeof(float4)));
    CK(cudaMalloc(&ctx->sorted, nsb));
    CK(cudaMalloc(&ctx->sbin, na * sizeof(int)));
    CK(cudaMalloc(&ctx->wrapv, na * sizeof(int)));
    CK(cudaMalloc(&ctx->atom_cell, na * sizeof(int)));
    CK(cudaMalloc(&ctx->atom_rank, na * sizeof(int)));
    CK(cudaMalloc(&ctx->atom_wrap, na * sizeof(int)));
    ctx->cap_atoms = na;
    ctx->cap_sorted_bytes = nsb;
  }
  if (ncell > ctx->cap_cells) {
    cudaFree(ctx->cell_count); cudaFree(ctx->cell_start); cudaFree(ctx->block_sums);
    ctx->cell_count = ctx->cell_start = ctx->block_sums = nullptr;
    ctx->cap_cells = 0;
    CK(cudaMalloc(&ctx->cell_count, (ncell + 1) * sizeof(int)));
    CK(cudaMalloc(&ctx->cell_start, (ncell + 1) * sizeof(int)));
    size_t nblk = (ncell + 1 + 2 * SCAN_BLOCK - 1) / (2 * SCAN_BLOCK);
    CK(cudaMalloc(&ctx->block_sums, (nblk + 1) * sizeof(int)));
    ctx->cap_cells = ncell;
  }
  return PTM_OK;
}

static bool finite_cell(const double *H) {
  for (int i = 0; i < 9; i++) if (!std::isfinite(H[i])) return false;
  return true;
}

// Output pointers of a frame descriptor.
static void set_outputs(FrameDesc *d, const ptm_outputs *o) {
  d->structure = o->structure; d->alloy = o->alloy; d->rmsd = o->rmsd; d->scale = o->scale;
  d->quat = o->quat; d->strain = o->strain; d->corr = o->correspondence;
  d->vm = o->von_mises; d->rf = o->rodrigues;
}

// Most cells a frame of n atoms is given (the cell grid is coarsened until it fits).
constexpr size_t max_cells(size_t n) { return 4 * n + 64; }

// Host description of one frame: its descriptor (device pointers are filled in
// by the caller once its workspace exists) and its binning parameters.  Shared
// by single frames, batches and the allocation-free entry.
static ptm_status setup_frame(const ptm_frame *f, double cell_factor, FrameDesc *desc, BinParams *bp,
                              size_t *ncell_out, ShiftTables *tab) {
  if (!f || f->n_atoms < 1 || f->n_atoms >= (1ll << 31) || !f->positions) return PTM_ERR_INVALID_ARG;
  if (f->ordering != PTM_ORDER_EUCLIDEAN && f->ordering != PTM_ORDER_TOPOLOGICAL) return PTM_ERR_INVALID_ARG;
  if (f->pos_dtype != PTM_F32 && f->pos_dtype != PTM_F64) return PTM_ERR_INVALID_ARG;
  if (!finite_cell(f->cell)) return PTM_ERR_INVALID_ARG;
  const double *H = f->cell;
  const double det = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                     H[2] * (H[3] * H[7] - H[4] * H[6]);
  if (!(std::fabs(det) > 1e-12)) return PTM_ERR_INVALID_ARG;
  const int64_t n = f->n_atoms;
  double Hinv[9], W[3];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
      Hinv[3 * i + j] = (H[3 * i1 + j1] * H[3 * i2 + j2] - H[3 * i1 + j2] * H[3 * i2 + j1]) / det;
    }
  for (int c = 0; c < 3; c++) W[c] = 1.0 / std::sqrt(Hinv[c] * Hinv[c] + Hinv[3 + c] * Hinv[3 + c] + Hinv[6 + c] * Hinv[6 + c]);
  const double rho = (double)n / std::fabs(det);
  const double wt = cell_factor * std::cbrt(3.0 * 15.0 / (4.0 * M_PI * rho));
  int nb[3];
  size_t ncell = 1;
  for (int c = 0; c < 3; c++) {
    nb[c] = std::min(std::max(1, (int)std::floor(W[c] / wt)), 1024);
    ncell *= (size_t)nb[c];
  }
  while (ncell > max_cells((size_t)n)) {
    int c = (int)(std::max_element(nb, nb + 3) - nb);
    ncell /= nb[c];
    nb[c] = std::max(1, nb[c] / 2);
    ncell *= nb[c];
  }
  std::memset(desc, 0, sizeof(FrameDesc));
  desc->species = f->species;
  desc->positions = f->positions;
  desc->n = n;
  for (int c = 0; c < 3; c++) { desc->nb[c] = nb[c]; desc->pbc[c] = f->pbc[c] ? 1 : 0; }
  desc->f64 = f->pos_dtype == PTM_F64;
  desc->ordering = f->ordering;
  desc->mask = f->template_mask ? (f->template_mask & PTM_MASK_ALL) : PTM_MASK_ALL;
  desc->rmsd_max = std::isnan(f->rmsd_max) ? INFINITY : (float)f->rmsd_max;
  desc->min_cell_width = (float)std::min(W[0] / nb[0], std::min(W[1] / nb[1], W[2] / nb[2]));
  for (int i = 0; i < 9; i++) desc->H[i] = H[i];
  // |n.H| for |n_r| <= 1 over the periodic rows r: at most the length of the
  // vector of per-component sums of |H_rc| (rounded up a little for FP32)
  double sm2 = 0.0;
  for (int k = 0; k < 3; k++) {
    double sk = 0.0;
    for (int r = 0; r < 3; r++) if (f->pbc[r]) sk += std::fabs(H[3 * r + k]);
    sm2 += sk * sk;
  }
  desc->smax = (float)(std::sqrt(sm2) * (1.0 + 1e-6));
  for (int a = -2; a <= 2; a++)
    for (int b = -2; b <= 2; b++)
      for (int c = -2; c <= 2; c++) {
        const int i = (a + 2) * 25 + (b + 2) * 5 + (c + 2);
        for (int k = 0; k < 3; k++) {
          volatile double t0 = (double)a * H[k];
          volatile double t1 = (double)b * H[3 + k];
          volatile double t2 = (double)c * H[6 + k];
          volatile double t01 = t0 + t1;
          const double sh = t01 + t2;
          tab->s64[i][k] = sh;
          tab->s32[i][k] = (float)sh;
          tab->slo[i][k] = (float)(sh - (double)(float)sh);
        }
      }
  std::memset(bp, 0, sizeof(BinParams));
  for (int i = 0; i < 9; i++) bp->Hinv[i] = (float)Hinv[i];
  for (int c = 0; c < 3; c++) { bp->W[c] = (float)W[c]; bp->nb[c] = nb[c]; bp->pbc[c] = desc->pbc[c]; }
  bp->n = n;
  bp->f64 = desc->f64;
  bp->pos = f->positions;
  *ncell_out = ncell;
  return PTM_OK;
}

// Enqueue the whole pipeline for one frame whose buffers are on the device.
static ptm_status enqueue_frame(ptm_context *ctx, const ptm_frame *f, const ptm_outputs *o, cudaStream_t st) {
  if (!f || !o) return PTM_ERR_INVALID_ARG;
  FrameDesc desc;
  BinParams bp;
  ShiftTables tab;
  size_t ncell = 0;
  ptm_status rs = setup_frame(f, 1.25, &desc, &bp, &ncell, &tab);
  if (rs != PTM_OK) return rs;
  const int64_t n = f->n_atoms;
  const int f64 = desc.f64;
  rs = grow(ctx, (size_t)n, ncell, f64);
  if (rs != PTM_OK) return rs;
  const bool topological = f->ordering == PTM_ORDER_TOPOLOGICAL;
  if ((size_t)n > ctx->cap_nbr) {
    cudaFree(ctx->nbr); cudaFree(ctx->lam); cudaFree(ctx->ents);
    ctx->nbr = nullptr; ctx->lam = nullptr; ctx->ents = nullptr;
    ctx->cap_nbr = 0;
    CK(cudaMalloc(&ctx->nbr, (size_t)n * PTM_KNN * sizeof(int2)));
    CK(cudaMalloc(&ctx->lam, (size_t)n * 3 * sizeof(uint64_t)));
    CK(cudaMalloc(&ctx->ents, (size_t)n * sizeof(uint32_t)));
    ctx->cap_nbr = (size_t)n;
  }
  if (topological && (size_t)n > ctx->cap_topo) {
    cudaFree(ctx->topo_list);
    cudaFree(ctx->topo_side);
    ctx->topo_list = nullptr;
    ctx->topo_side = nullptr;
    ctx->cap_topo = 0;
    CK(cudaMalloc(&ctx->topo_list, ((size_t)n + 1) * sizeof(int)));
    CK(cudaMalloc(&ctx->topo_side, topo_side_bytes((size_t)n)));
    ctx->cap_topo = (size_t)n;
  }
  desc.sorted = ctx->sorted;
  desc.sbin = ctx->sbin;
  desc.cell_start = ctx->cell_start;
  desc.wrapv = ctx->wrapv;
  set_outputs(&desc, o);
  desc.dstat = ctx->dstat;
  desc.counters = ctx->counters;
  desc.nbr = ctx->nbr;
  desc.lam = ctx->lam;
  desc.ents = ctx->ents;
  desc.tab = ctx->tab;
  bp.counters = ctx->counters;

  cudaGetLastError();   // launch errors are read below; drop any left by earlier calls
  CK(cudaEventRecord(ctx->ev[0], st));
  CK(cudaMemsetAsync(ctx->cell_count, 0, (ncell + 1) * sizeof(int), st));
  CK(cudaMemsetAsync(ctx->dstat, 0, 4 * sizeof(int), st));
  CK(cudaMemsetAsync(ctx->counters, 0, C_NCOUNTERS * sizeof(unsigned long long), st));
  k_put_tables<<<1, 256, 0, st>>>(tab, ctx->tab);
  const int tb = 256;
  const unsigned gb = (unsigned)((n + tb - 1) / tb);
  k_bin<<<gb, tb, 0, st>>>(f->positions, bp, ctx->cell_count, ctx->atom_cell, ctx->atom_rank, ctx->atom_wrap,
                           ctx->dstat);
  const int nscan = (int)ncell + 1;
  const int nblk = (nscan + 2 * SCAN_BLOCK - 1) / (2 * SCAN_BLOCK);
  k_scan_block<<<nblk, SCAN_BLOCK, 0, st>>>(ctx->cell_count, ctx->cell_start, ctx->block_sums, nscan);
  k_scan_sums<<<1, SCAN_BLOCK, 0, st>>>(ctx->block_sums, nblk, ctx->dstat + 2);
  k_scan_add<<<(nscan + 255) / 256, 256, 0, st>>>(ctx->cell_start, ctx->block_sums, nscan);
  k_scatter<<<gb, tb, 0, st>>>(f->positions, f64, n, ctx->atom_cell, ctx->atom_rank, ctx->atom_wrap,
                               ctx->cell_start, ctx->sorted, ctx->sbin, ctx->wrapv);
  const unsigned ga = (unsigned)((n + PTM_BLOCK - 1) / PTM_BLOCK);
  CK(cudaEventRecord(ctx->ev[1], st));
  if (!topological) {
    const unsigned gk = (unsigned)((n + PTM_KNN_BLOCK - 1) / PTM_KNN_BLOCK);
    if (f64) k_knn<true><<<gk, PTM_KNN_BLOCK, knn_smem_bytes(), st>>>(desc);
    else k_knn<false><<<gk, PTM_KNN_BLOCK, knn_smem_bytes(), st>>>(desc);
  } else {
    int *cnt = ctx->topo_list + ctx->cap_topo;
    CK(cudaMemsetAsync(cnt, 0, sizeof(int), st));
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    const int cap_side = (int)topo_side_cap(ctx->cap_topo);
    const unsigned g64 = (unsigned)(PTM_TOPO64_BLOCKS_PER_SM * sms);
    if (f64) {
      k_topo<true><<<ga, PTM_BLOCK, topo_smem_bytes(), st>>>(desc, ctx->nbr, ctx->topo_list, cnt, ctx->topo_side,
                                                             cap_side);
      k_topo64<true><<<g64, PTM_BLOCK, topo64_smem_bytes(), st>>>(desc, ctx->nbr, ctx->topo_list, cnt,
                                                                  ctx->topo_side, cap_side);
    } else {
      k_topo<false><<<ga, PTM_BLOCK, topo_smem_bytes(), st>>>(desc, ctx->nbr, ctx->topo_list, cnt, ctx->topo_side,
                                                              cap_side);
      k_topo64<false><<<g64, PTM_BLOCK, topo64_smem_bytes(), st>>>(desc, ctx->nbr, ctx->topo_list, cnt,
                                                                   ctx->topo_side, cap_side);
    }
  }
  CK(cudaEventRecord(ctx->ev[3], st));
  if (f64) k_hulls<true><<<ga, PTM_BLOCK, atom_smem_bytes(), st>>>(desc);
  else k_hulls<false><<<ga, PTM_BLOCK, atom_smem_bytes(), st>>>(desc);
  CK(cudaEventRecord(ctx->ev[4], st));
  if (ctx->precision == PTM_PREC_FP64) {
    if (f64) k_match<true, true><<<ga, PTM_BLOCK, match_smem_bytes(), st>>>(desc);
    else k_match<false, true><<<ga, PTM_BLOCK, match_smem_bytes(), st>>>(desc);
  } else {
    if (f64) k_match<true><<<ga, PTM_BLOCK, match_smem_bytes(), st>>>(desc);
    else k_match<false><<<ga, PTM_BLOCK, match_smem_bytes(), st>>>(desc);
  }
  CK(cudaGetLastError());
  CK(cudaEventRecord(ctx->ev[2], st));
  ctx->last_stream = st;
  // k_put_tables, k_bin, three scans, k_scatter, k_knn or k_topo + k_topo64, k_hulls, k_match
  ctx->launches = topological ? 10 : 9;
  return PTM_OK;
}

extern "C" {

const char *ptm_status_string(ptm_status s) {
  switch (s) {
    case PTM_OK: return "PTM_OK";
    case PTM_ERR_INVALID_ARG: return "PTM_ERR_INVALID_ARG";
    case PTM_ERR_OUT_OF_MEMORY: return "PTM_ERR_OUT_OF_MEMORY";
    case PTM_ERR_CUDA: return "PTM_ERR_CUDA";
    case PTM_ERR_TIMEOUT: return "PTM_ERR_TIMEOUT";
    case PTM_ERR_DEVICE_STATUS: return "PTM_ERR_DEVICE_STATUS";
    case PTM_ERR_BUSY: return "PTM_ERR_BUSY";
    case PTM_ERR_NOT_FOUND: return "PTM_ERR_NOT_FOUND";
  }
  return "PTM_ERR_UNKNOWN";
}

const char *ptm_last_cuda_error(ptm_context *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

ptm_status ptm_create(const ptm_options *opt, ptm_context **out) {
  if (!out) return PTM_ERR_INVALID_ARG;
  *out = nullptr;
  ptm_context *ctx = new (std::nothrow) ptm_context();
  if (!ctx) return PTM_ERR_OUT_OF_MEMORY;
  ctx->device = opt ? opt->device : 0;
  ctx->precision = opt ? opt->precision : PTM_PREC_FP32;
  if (ctx->precision != PTM_PREC_FP32 && ctx->precision != PTM_PREC_FP64) { delete ctx; return PTM_ERR_INVALID_ARG; }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ctx->device < 0 || ctx->device >= ndev) {
    delete ctx;
    return e != cudaSuccess ? PTM_ERR_CUDA : PTM_ERR_INVALID_ARG;
  }
  ptm_status rs = PTM_OK;
  do {
    if ((e = cudaSetDevice(ctx->device)) != cudaSuccess) { rs = cuda_fail(ctx, e, "cudaSetDevice"); break; }
    if ((e = cudaMalloc(&ctx->dstat, 8 * sizeof(int))) != cudaSuccess) { rs = cuda_fail(ctx, e, "cudaMalloc"); break; }
    if ((e = cudaMalloc(&ctx->counters, C_NCOUNTERS * sizeof(unsigned long long))) != cudaSuccess) { rs = cuda_fail(ctx, e, "cudaMalloc"); break; }
    if ((e = cudaMalloc(&ctx->tab, sizeof(ShiftTables))) != cudaSuccess) { rs = cuda_fail(ctx, e, "cudaMalloc"); break; }
    for (int i = 0; i < 5 && e == cudaSuccess; i++) e = cudaEventCreate(&ctx->ev[i]);
    if (e != cudaSuccess) { rs = cuda_fail(ctx, e, "cudaEventCreate"); break; }
    if ((e = cudaMemset(ctx->counters, 0, C_NCOUNTERS * sizeof(unsigned long long))) != cudaSuccess) { rs = cuda_fail(ctx, e, "cudaMemset"); break; }
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    ctx->budget = (opt && opt->hbm_budget_bytes) ? opt->hbm_budget_bytes : fr / 2;
    // the per-atom kernels want every resident block's scratch in shared
    // memory: the largest shared-memory carveout of the unified L1
    const int smem = (int)std::max(atom_smem_bytes(), std::max(topo_smem_bytes(), topo64_smem_bytes()));
    const void *fns[] = {(const void *)k_hulls<false>, (const void *)k_hulls<true>, (const void *)k_hulls_batch<false>,
                         (const void *)k_hulls_batch<true>, (const void *)k_match<false>, (const void *)k_match<true>,
                         (const void *)k_match<false, true>, (const void *)k_match<true, true>,
                         (const void *)k_match_batch<false>, (const void *)k_match_batch<true>,
                         (const void *)k_topo<false>, (const void *)k_topo<true>,
                         (const void *)k_topo_batch<false>, (const void *)k_topo_batch<true>,
                         (const void *)k_topo64<false>, (const void *)k_topo64<true>,
                         (const void *)k_topo64_batch<false>, (const void *)k_topo64_batch<true>,
                         (const void *)k_knn<false>, (const void *)k_knn<true>, (const void *)k_knn_batch<false>,
                         (const void *)k_knn_batch<true>};
    for (const void *fn : fns) {
      if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess ||
          (e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
        break;
    }
    if (e != cudaSuccess) { rs = cuda_fail(ctx, e, "cudaFuncSetAttribute"); break; }
  } while (0);
  if (rs != PTM_OK) { ptm_destroy(ctx); return rs; }
  *out = ctx;
  return PTM_OK;
}

ptm_status ptm_destroy(ptm_context *ctx) {
  if (!ctx) return PTM_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  cudaFree(ctx->sorted); cudaFree(ctx->sbin); cudaFree(ctx->wrapv);
  cudaFree(ctx->atom_cell); cudaFree(ctx->atom_rank); cudaFree(ctx->atom_wrap);
  cudaFree(ctx->cell_count); cudaFree(ctx->cell_start); cudaFree(ctx->block_sums);
  cudaFree(ctx->dstat); cudaFree(ctx->counters); cudaFree(ctx->tab);
  for (int i = 0; i < 5; i++) if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  cudaFree(ctx->hpos); cudaFree(ctx->hspecies);
  cudaFree(ctx->o_struct); cudaFree(ctx->o_alloy); cudaFree(ctx->o_rmsd); cudaFree(ctx->o_scale);
  cudaFree(ctx->o_quat); cudaFree(ctx->o_strain); cudaFree(ctx->o_corr); cudaFree(ctx->o_vm); cudaFree(ctx->o_rf);
  cudaFree(ctx->nbr); cudaFree(ctx->lam); cudaFree(ctx->ents);
  cudaFree(ctx->topo_list);
  cudaFree(ctx->topo_side);
  delete ctx;
  return PTM_OK;
}

ptm_status ptm_classify_frame(ptm_context *ctx, const ptm_frame *frame, const ptm_outputs *out, void *stream) {
  if (!ctx) return PTM_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  return enqueue_frame(ctx, frame, out, (cudaStream_t)stream);
}

ptm_status ptm_classify_frame_host(ptm_context *ctx, const ptm_frame *frame, const ptm_outputs *out,
                                   void *stream) {
  if (!ctx || !frame || !out) return PTM_ERR_INVALID_ARG;
  if (frame->n_atoms < 1 || frame->n_atoms >= (1ll << 31) || !frame->positions) return PTM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaSetDevice(ctx->device));
  const size_t n = (size_t)frame->n_atoms;
  const size_t esz = frame->pos_dtype == PTM_F64 ? 8 : 4;
  if (n > ctx->cap_host_atoms) {
    cudaFree(ctx->hpos); cudaFree(ctx->hspecies);
    cudaFree(ctx->o_struct); cudaFree(ctx->o_alloy); cudaFree(ctx->o_rmsd); cudaFree(ctx->o_scale);
    cudaFree(ctx->o_quat); cudaFree(ctx->o_strain); cudaFree(ctx->o_corr); cudaFree(ctx->o_vm); cudaFree(ctx->o_rf);
    ctx->hpos = nullptr; ctx->hspecies = nullptr; ctx->o_struct = ctx->o_alloy = nullptr;
    ctx->o_rmsd = ctx->o_scale = ctx->o_quat = ctx->o_strain = nullptr; ctx->o_corr = nullptr;
    ctx->o_vm = ctx->o_rf = nullptr;
    ctx->cap_host_atoms = 0;
    CK(cudaMalloc(&ctx->hpos, n * 3 * 8));
    CK(cudaMalloc(&ctx->hspecies, n));
    CK(cudaMalloc(&ctx->o_struct, n));
    CK(cudaMalloc(&ctx->o_alloy, n));
    CK(cudaMalloc(&ctx->o_rmsd, n * 4));
    CK(cudaMalloc(&ctx->o_scale, n * 4));
    CK(cudaMalloc(&ctx->o_quat, n * 16));
    CK(cudaMalloc(&ctx->o_strain, n * 36));
    CK(cudaMalloc(&ctx->o_corr, n * 60));
    CK(cudaMalloc(&ctx->o_vm, n * 4));
    CK(cudaMalloc(&ctx->o_rf, n * 12));
    ctx->cap_host_atoms = n;
  }
  CK(cudaMemcpyAsync(ctx->hpos, frame->positions, n * 3 * esz, cudaMemcpyHostToDevice, st));
  if (frame->species) CK(cudaMemcpyAsync(ctx->hspecies, frame->species, n, cudaMemcpyHostToDevice, st));
  ptm_frame df = *frame;
  df.positions = ctx->hpos;
  df.species = frame->species ? ctx->hspecies : nullptr;
  ptm_outputs dout;
  dout.structure = out->structure ? ctx->o_struct : nullptr;
  dout.alloy = out->alloy ? ctx->o_alloy : nullptr;
  dout.rmsd = out->rmsd ? ctx->o_rmsd : nullptr;
  dout.scale = out->scale ? ctx->o_scale : nullptr;
  dout.quat = out->quat ? ctx->o_quat : nullptr;
  dout.strain = out->strain ? ctx->o_strain : nullptr;
  dout.correspondence = out->correspondence ? ctx->o_corr : nullptr;
  dout.von_mises = out->von_mises ? ctx->o_vm : nullptr;
  dout.rodrigues = out->rodrigues ? ctx->o_rf : nullptr;
  ptm_status rs = enqueue_frame(ctx, &df, &dout, st);
  if (rs != PTM_OK) return rs;
  if (out->structure) CK(cudaMemcpyAsync(out->structure, dout.structure, n, cudaMemcpyDeviceToHost, st));
  if (out->alloy) CK(cudaMemcpyAsync(out->alloy, dout.alloy, n, cudaMemcpyDeviceToHost, st));
  if (out->rmsd) CK(cudaMemcpyAsync(out->rmsd, dout.rmsd, n * 4, cudaMemcpyDeviceToHost, st));
  if (out->scale) CK(cudaMemcpyAsync(out->scale, dout.scale, n * 4, cudaMemcpyDeviceToHost, st));
  if (out->quat) CK(cudaMemcpyAsync(out->quat, dout.quat, n * 16, cudaMemcpyDeviceToHost, st));
  if (out->strain) CK(cudaMemcpyAsync(out->strain, dout.strain, n * 36, cudaMemcpyDeviceToHost, st));
  if (out->correspondence) CK(cudaMemcpyAsync(out->correspondence, dout.correspondence, n * 60, cudaMemcpyDeviceToHost, st));
  if (out->von_mises) CK(cudaMemcpyAsync(out->von_mises, dout.von_mises, n * 4, cudaMemcpyDeviceToHost, st));
  if (out->rodrigues) CK(cudaMemcpyAsync(out->rodrigues, dout.rodrigues, n * 12, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return PTM_OK;
}

ptm_status ptm_get_stats(ptm_context *ctx, ptm_stats *out) {
  if (!ctx || !out) return PTM_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->last_stream));
  unsigned long long c[C_NCOUNTERS];
  CK(cudaMemcpy(c, ctx->counters, sizeof c, cudaMemcpyDeviceToHost));
  float t_all = 0.f, t_atom = 0.f;
  if (cudaEventElapsedTime(&t_all, ctx->ev[0], ctx->ev[2]) != cudaSuccess) t_all = -1.f;
  if (cudaEventElapsedTime(&t_atom, ctx->ev[1], ctx->ev[2]) != cudaSuccess) t_atom = -1.f;
  float t_cls = -1.f, t_match = -1.f;
  if (cudaEventElapsedTime(&t_cls, ctx->ev[3], ctx->ev[2]) != cudaSuccess) t_cls = -1.f;
  if (cudaEventElapsedTime(&t_match, ctx->ev[4], ctx->ev[2]) != cudaSuccess) t_match = -1.f;
  cudaGetLastError();
  out->pipeline_ms = t_all;
  out->atom_kernel_ms = t_atom;
  out->classify_kernel_ms = t_cls;
  out->match_kernel_ms = t_match;
  out->kernel_launches = ctx->launches;
  out->candidates = (int64_t)c[C_CAND];
  out->candidate_points = (int64_t)c[C_CANDPTS];
  out->atoms = (int64_t)c[C_ATOMS];
  out->matched = (int64_t)c[C_MATCHED];
  out->knn_wide = (int64_t)c[C_KNN_WIDE];
  out->knn_fail = (int64_t)c[C_KNN_FAIL];
  out->sos = (int64_t)c[C_SOS];
  out->qcp_fp64 = (int64_t)c[C_QCP64];
  out->tie_fp64 = (int64_t)c[C_TIE64];
  out->topo_fp64 = (int64_t)c[C_TOPO64];
  out->knn_fp64 = (int64_t)c[C_KNN64];
  out->excluded = (int64_t)c[C_EXCLUDED];
  out->internal = (int64_t)c[C_INTERNAL];
  return PTM_OK;
}

}  // extern "C"

// ================================================================== batches
struct ptm_batch {
  ptm_context *ctx = nullptr;
  int nframes = 0, f64 = 0;
  int64_t ntotal = 0;
  size_t ncell = 0;
  int tile_atoms = 32, blocks_per_sm = PTM_ATOM_BLOCKS_PER_SM;
  double cell_factor = 1.25;
  FrameDesc *d_descs = nullptr;
  ShiftTables *d_tabs = nullptr;
  BinParams *d_bp = nullptr;
  int64_t *d_atom_off = nullptr;
  int *d_dstat = nullptr;
  void *sorted = nullptr;
  int *sbin = nullptr, *wrapv = nullptr, *atom_cell = nullptr, *atom_rank = nullptr, *atom_wrap = nullptr;
  int *cell_count = nullptr, *cell_start = nullptr, *block_sums = nullptr, *scan_total = nullptr;
  unsigned long long *queue = nullptr, *counters = nullptr;
  cudaEvent_t ev[5] = {};       // as ptm_context::ev
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int nsm = 152;
  int topo = 0;                   // some frame takes the topological order
  int2 *nbr_buf = nullptr;        // per-frame segments of neighbour lists
  uint64_t *lam_buf = nullptr;    // per-frame segments of the k_hulls -> k_match state
  uint32_t *ents_buf = nullptr;
  std::vector<FrameDesc> own;     // frames with a k_match launch of their own (PTM_MATCH_OWN_LAUNCH)
  int nsmall = 0;                 // the other frames: one persistent k_match_batch over their atoms
  int64_t small_atoms = 0;
  int *d_small_frames = nullptr;
  int64_t *d_small_off = nullptr;
  int launches = 0;               // kernels the last enqueue launched
  cudaStream_t side[PTM_MATCH_SIDE_STREAMS] = {};   // the own k_match launches fork onto these
  cudaEvent_t fork = nullptr, join[PTM_MATCH_SIDE_STREAMS] = {};
  int nside = 0;
  int *topo_list = nullptr;       // atoms for the FP64 pass; [ntotal] = their count
  TopoSide *topo_side = nullptr;  // what the FP32 pass keeps for the FP64 pass
  void *block = nullptr;          // the workspace (one allocation, or a pool block when served)
  bool owns_block = true;
};

static void batch_free(ptm_batch *b) {
  if (!b) return;
  for (int i = 0; i < b->nside; i++) {
    if (b->join[i]) cudaEventDestroy(b->join[i]);
    if (b->side[i]) cudaStreamDestroy(b->side[i]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->owns_block) cudaFree(b->block);
  for (int i = 0; i < 5; i++) if (b->ev[i]) cudaEventDestroy(b->ev[i]);
  delete b;
}

// Side streams and fork / join events for a batch with two or more own
// k_match launches (created outside any stream capture).
static cudaError_t batch_side_init(ptm_batch *b) {
  const int want = (int)std::min<size_t>(PTM_MATCH_SIDE_STREAMS, b->own.size() > 1 ? b->own.size() - 1 : 0);
  cudaError_t e = cudaSuccess;
  if (want && !b->fork) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < want && e == cudaSuccess; i++) {
    e = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    if (e == cudaSuccess) b->nside = i + 1;
  }
  return e;
}

// Enqueue one pass over the whole batch: binning of every frame, one scan over
// all cells, scatter, then the persistent classification launch.
static ptm_status batch_enqueue(ptm_batch *b, cudaStream_t st) {
  ptm_context *ctx = b->ctx;
  cudaGetLastError();   // launch errors are read below; drop any left by earlier calls
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cap));
  const unsigned rec = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  CK(cudaEventRecordWithFlags(b->ev[0], st, rec));
  CK(cudaMemsetAsync(b->cell_count, 0, (b->ncell + 1) * sizeof(int), st));
  CK(cudaMemsetAsync(b->d_dstat, 0, (size_t)4 * b->nframes * sizeof(int), st));
  CK(cudaMemsetAsync(b->counters, 0, C_NCOUNTERS * sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(b->queue, 0, 2 * sizeof(unsigned long long), st));
  const int tb = 256;
  const unsigned gb = (unsigned)((b->ntotal + tb - 1) / tb);
  k_bin_batch<<<gb, tb, 0, st>>>(b->d_bp, b->d_atom_off, b->nframes, b->ntotal, b->cell_count, b->atom_cell,
                                 b->atom_rank, b->atom_wrap);
  const int nscan = (int)b->ncell + 1;
  const int nblk = (nscan + 2 * SCAN_BLOCK - 1) / (2 * SCAN_BLOCK);
  k_scan_block<<<nblk, SCAN_BLOCK, 0, st>>>(b->cell_count, b->cell_start, b->block_sums, nscan);
  k_scan_sums<<<1, SCAN_BLOCK, 0, st>>>(b->block_sums, nblk, b->scan_total);
  k_scan_add<<<(nscan + 255) / 256, 256, 0, st>>>(b->cell_start, b->block_sums, nscan);
  k_scatter_batch<<<gb, tb, 0, st>>>(b->d_bp, b->d_atom_off, b->nframes, b->ntotal, b->atom_cell, b->atom_rank,
                                     b->atom_wrap, b->cell_start, b->sorted, b->sbin, b->wrapv);
  CK(cudaEventRecordWithFlags(b->ev[1], st, rec));
  if (b->topo != 2) {           // some frame takes the Euclidean order
    const unsigned gk = (unsigned)((b->ntotal + PTM_KNN_BLOCK - 1) / PTM_KNN_BLOCK);
    if (b->f64)
      k_knn_batch<true><<<gk, PTM_KNN_BLOCK, knn_smem_bytes(), st>>>(b->d_descs, b->d_atom_off, b->nframes, b->ntotal);
    else
      k_knn_batch<false><<<gk, PTM_KNN_BLOCK, knn_smem_bytes(), st>>>(b->d_descs, b->d_atom_off, b->nframes, b->ntotal);
  }
  if (b->topo) {
    int *cnt = b->topo_list + b->ntotal;
    CK(cudaMemsetAsync(cnt, 0, sizeof(int), st));
    const unsigned gt = (unsigned)((b->ntotal + PTM_BLOCK - 1) / PTM_BLOCK);
    const int cap_side = (int)topo_side_cap((size_t)b->ntotal);
    const unsigned g64 = (unsigned)(PTM_TOPO64_BLOCKS_PER_SM * b->nsm);
    if (b->f64) {
      k_topo_batch<true><<<gt, PTM_BLOCK, topo_smem_bytes(), st>>>(b->d_descs, b->d_atom_off, b->nframes, b->ntotal,
                                                                 b->topo_list, cnt, b->topo_side, cap_side);
      k_topo64_batch<true><<<g64, PTM_BLOCK, topo64_smem_bytes(), st>>>(b->d_descs, b->d_atom_off, b->nframes,
                                                                        b->topo_list, cnt, b->topo_side, cap_side);
    } else {
      k_topo_batch<false><<<gt, PTM_BLOCK, topo_smem_bytes(), st>>>(b->d_descs, b->d_atom_off, b->nframes, b->ntotal,
                                                                  b->topo_list, cnt, b->topo_side, cap_side);
      k_topo64_batch<false><<<g64, PTM_BLOCK, topo64_smem_bytes(), st>>>(b->d_descs, b->d_atom_off, b->nframes,
                                                                         b->topo_list, cnt, b->topo_side, cap_side);
    }
  }
  CK(cudaEventRecordWithFlags(b->ev[3], st, rec));
  // persistent grids: two warps per block, each pulling its own tiles
  const int64_t tiles = (b->ntotal + b->tile_atoms - 1) / b->tile_atoms;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)b->nsm * b->blocks_per_sm,
                                                                       (tiles + 1) / 2));
  if (b->f64)
    k_hulls_batch<true><<<grid, PTM_BLOCK, atom_smem_bytes(), st>>>(b->d_descs, b->d_atom_off, b->nframes,
                                                                    b->ntotal, b->tile_atoms, b->queue);
  else
    k_hulls_batch<false><<<grid, PTM_BLOCK, atom_smem_bytes(), st>>>(b->d_descs, b->d_atom_off, b->nframes,
                                                                     b->ntotal, b->tile_atoms, b->queue);
  CK(cudaEventRecordWithFlags(b->ev[4], st, rec));
  // the frames' own k_match launches alternate between the batch stream and
  // the side streams, so that one launch's last wave overlaps the next launch
  const int ns = b->nside;
  if (ns) {
    CK(cudaEventRecord(b->fork, st));
    for (int i = 0; i < ns; i++) CK(cudaStreamWaitEvent(b->side[i], b->fork, 0));
  }
  for (size_t k = 0; k < b->own.size(); k++) {
    const FrameDesc &hd = b->own[k];
    const int w = (int)(k % (size_t)(ns + 1));
    cudaStream_t sk = w == 0 ? st : b->side[w - 1];
    const unsigned g = (unsigned)((hd.n + PTM_BLOCK - 1) / PTM_BLOCK);
    if (b->f64) k_match<true><<<g, PTM_BLOCK, match_smem_bytes(), sk>>>(hd);
    else k_match<false><<<g, PTM_BLOCK, match_smem_bytes(), sk>>>(hd);
  }
  if (b->nsmall) {
    const int64_t stiles = (b->small_atoms + b->tile_atoms - 1) / b->tile_atoms;
    const unsigned grid_m = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)b->nsm * PTM_MATCH_BLOCKS_PER_SM, (stiles + 1) / 2));
    if (b->f64)
      k_match_batch<true><<<grid_m, PTM_BLOCK, match_smem_bytes(), st>>>(b->d_descs, b->d_small_off, b->d_small_frames,
                                                                         b->nsmall, b->small_atoms, b->tile_atoms,
                                                                         b->queue + 1);
    else
      k_match_batch<false><<<grid_m, PTM_BLOCK, match_smem_bytes(), st>>>(b->d_descs, b->d_small_off,
                                                                          b->d_small_frames, b->nsmall, b->small_atoms,
                                                                          b->tile_atoms, b->queue + 1);
  }
  if (ns) {
    for (int i = 0; i < ns; i++) {
      CK(cudaEventRecord(b->join[i], b->side[i]));
      CK(cudaStreamWaitEvent(st, b->join[i], 0));
    }
  }
  b->launches = 7 + (b->topo ? 2 : 0) + (int)b->own.size() + (b->nsmall ? 1 : 0) - (b->topo == 2 ? 1 : 0);
  CK(cudaGetLastError());
  CK(cudaEventRecordWithFlags(b->ev[2], st, rec));
  return PTM_OK;
}

// Host-side preparation of a batch: descriptors, binning parameters and
// offsets of every frame, total atoms and cells.
struct BatchPlan {
  std::vector<FrameDesc> hd;
  std::vector<ShiftTables> tabs;
  std::vector<BinParams> hb;
  std::vector<int64_t> off;
  int64_t ntotal = 0;
  size_t ncell = 0;
  int f64 = 0;
  int topo = 0;                      // 0: no frame, 1: some, 2: every frame in the topological order
  int ntopo = 0;
  std::vector<int> ordering;
  std::vector<int> small_frames;     // frames below PTM_MATCH_OWN_LAUNCH atoms ...
  std::vector<int64_t> small_off;    // ... and the prefix sum of their sizes
  int64_t small_atoms = 0;
};

static ptm_status batch_plan(int nframes, const ptm_frame *frames, double cell_factor, BatchPlan &P) {
  P.hd.resize(nframes);
  P.tabs.resize(nframes);
  P.hb.resize(nframes);
  P.off.resize(nframes);
  P.ordering.resize(nframes);
  P.f64 = frames[0].pos_dtype == PTM_F64;
  for (int f = 0; f < nframes; f++) {
    size_t nc = 0;
    ptm_status rs = setup_frame(&frames[f], cell_factor, &P.hd[f], &P.hb[f], &nc, &P.tabs[f]);
    if (rs == PTM_OK && (frames[f].pos_dtype == PTM_F64) != (P.f64 != 0)) rs = PTM_ERR_INVALID_ARG;
    if (rs != PTM_OK) return rs;
    P.off[f] = P.ntotal;
    P.hb[f].atom_off = P.ntotal;
    P.hb[f].cell_off = (int)P.ncell;
    P.hd[f].atom_offset = P.ntotal;
    P.ordering[f] = frames[f].ordering;
    P.ntopo += frames[f].ordering == PTM_ORDER_TOPOLOGICAL;
    P.ntotal += frames[f].n_atoms;
    P.ncell += nc;
    if (P.ntotal >= (1ll << 31) || P.ncell >= (1ull << 31)) return PTM_ERR_INVALID_ARG;
  }
  P.topo = P.ntopo == 0 ? 0 : (P.ntopo == nframes ? 2 : 1);
  for (int f = 0; f < nframes; f++)
    if (frames[f].n_atoms < PTM_MATCH_OWN_LAUNCH) {
      P.small_frames.push_back(f);
      P.small_off.push_back(P.small_atoms);
      P.small_atoms += frames[f].n_atoms;
    }
  return PTM_OK;
}

// Device bytes of a batch's workspace (descriptors, sorted atoms, cell lists).
static size_t batch_workspace_bytes(int nframes, int64_t ntotal, size_t ncell, int f64, int topo) {
  const size_t n = (size_t)ntotal, rec = f64 ? sizeof(Atom64) : sizeof(float4);
  const size_t nblk = (ncell + 1 + 2 * SCAN_BLOCK - 1) / (2 * SCAN_BLOCK) + 1;
  const size_t tb = sizeof(int2) * PTM_KNN * n + 28 * n + 3 * 256 +
                    (topo ? 4 * (n + 1) + topo_side_bytes(n) + 2 * 256 : 0);
  return (sizeof(FrameDesc) + sizeof(ShiftTables) + sizeof(BinParams) + 2 * sizeof(int64_t) + sizeof(int) + 16) *
             nframes + 3 * 256 +
         rec * n + 20 * n +
         8 * (ncell + 1) + 4 * nblk + 4 + 16 + 8 * C_NCOUNTERS + 16 * 256 + tb;
}

// Carve the batch workspace out of one device block (256-byte aligned pieces)
// and point the descriptors at it.
static void batch_layout(ptm_batch *b, unsigned char *base, BatchPlan &P, const ptm_outputs *outs) {
  size_t o = 0;
  auto take = [&](size_t bytes) { void *p = base + o; o += (bytes + 255) / 256 * 256; return p; };
  const size_t n = (size_t)P.ntotal, nc = P.ncell;
  const size_t nblk = (nc + 1 + 2 * SCAN_BLOCK - 1) / (2 * SCAN_BLOCK) + 1;
  const int nf = b->nframes;
  b->d_descs = (FrameDesc *)take(sizeof(FrameDesc) * nf);
  b->d_tabs = (ShiftTables *)take(sizeof(ShiftTables) * nf);
  b->d_bp = (BinParams *)take(sizeof(BinParams) * nf);
  b->d_small_frames = (int *)take(sizeof(int) * nf);
  b->d_small_off = (int64_t *)take(sizeof(int64_t) * nf);
  b->d_atom_off = (int64_t *)take(sizeof(int64_t) * nf);
  b->d_dstat = (int *)take(sizeof(int) * 4 * nf);
  b->sorted = take((P.f64 ? sizeof(Atom64) : sizeof(float4)) * n);
  b->sbin = (int *)take(4 * n); b->wrapv = (int *)take(4 * n); b->atom_cell = (int *)take(4 * n);
  b->atom_rank = (int *)take(4 * n); b->atom_wrap = (int *)take(4 * n);
  b->cell_count = (int *)take(4 * (nc + 1)); b->cell_start = (int *)take(4 * (nc + 1));
  b->block_sums = (int *)take(4 * nblk); b->scan_total = (int *)take(4);
  b->queue = (unsigned long long *)take(16); b->counters = (unsigned long long *)take(8 * C_NCOUNTERS);
  b->topo = P.topo;
  b->nbr_buf = (int2 *)take(sizeof(int2) * PTM_KNN * n);
  b->lam_buf = (uint64_t *)take(sizeof(uint64_t) * 3 * n);
  b->ents_buf = (uint32_t *)take(sizeof(uint32_t) * n);
  if (P.topo) {
    b->topo_list = (int *)take(4 * (n + 1));
    b->topo_side = (TopoSide *)take(topo_side_bytes(n));
  }
  for (int f = 0; f < nf; f++) {
    // frame f's neighbour list: rows of n_f entries from slot 14 x (first slot)
    P.hd[f].nbr = b->nbr_buf + PTM_KNN * P.off[f];
    P.hd[f].lam = b->lam_buf + 3 * P.off[f];
    P.hd[f].ents = b->ents_buf + P.off[f];
    P.hd[f].tab = b->d_tabs + f;
    P.hd[f].sorted = b->sorted;
    P.hd[f].sbin = b->sbin;
    P.hd[f].cell_start = b->cell_start + P.hb[f].cell_off;
    P.hd[f].wrapv = b->wrapv;
    set_outputs(&P.hd[f], &outs[f]);
    P.hd[f].dstat = b->d_dstat + 4 * f;
    P.hd[f].counters = b->counters;
    P.hb[f].dstat = b->d_dstat + 4 * f;
    P.hb[f].counters = b->counters;
  }
  b->own.clear();
  for (int f = 0; f < nf; f++) if (P.hd[f].n >= PTM_MATCH_OWN_LAUNCH) b->own.push_back(P.hd[f]);
  b->nsmall = (int)P.small_frames.size();
  b->small_atoms = P.small_atoms;
}

extern "C" ptm_status ptm_batch_create(ptm_context *ctx, int nframes, const ptm_frame *frames, const ptm_outputs *outs,
                                       const ptm_tuning *tuning, ptm_batch **out) {
  if (!ctx || !frames || !outs || !out || nframes < 1) return PTM_ERR_INVALID_ARG;
  *out = nullptr;
  CK(cudaSetDevice(ctx->device));
  ptm_batch *b = new (std::nothrow) ptm_batch();
  if (!b) return PTM_ERR_OUT_OF_MEMORY;
  b->ctx = ctx;
  b->nframes = nframes;
  if (tuning) {
    if (tuning->cell_factor > 0) b->cell_factor = tuning->cell_factor;
    if (tuning->tile_atoms > 0) b->tile_atoms = (tuning->tile_atoms + 31) / 32 * 32;
    if (tuning->blocks_per_sm > 0) b->blocks_per_sm = tuning->blocks_per_sm;
  }
  if (!(b->cell_factor >= 0.5 && b->cell_factor <= 4.0)) { delete b; return PTM_ERR_INVALID_ARG; }
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  BatchPlan P;
  ptm_status rs = batch_plan(nframes, frames, b->cell_factor, P);
  if (rs != PTM_OK) { delete b; return rs; }
  b->f64 = P.f64;
  b->ntotal = P.ntotal;
  b->ncell = P.ncell;
  cudaError_t e = cudaMalloc(&b->block, batch_workspace_bytes(nframes, P.ntotal, P.ncell, P.f64, P.topo));
  for (int i = 0; i < 5 && e == cudaSuccess; i++) e = cudaEventCreate(&b->ev[i]);
  if (e != cudaSuccess) { rs = cuda_fail(ctx, e, "ptm_batch_create"); batch_free(b); return rs; }
  batch_layout(b, (unsigned char *)b->block, P, outs);
  if ((e = batch_side_init(b)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_descs, P.hd.data(), sizeof(FrameDesc) * nframes, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_tabs, P.tabs.data(), sizeof(ShiftTables) * nframes, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (b->nsmall && (e = cudaMemcpy(b->d_small_frames, P.small_frames.data(), sizeof(int) * b->nsmall,
                                    cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (b->nsmall && (e = cudaMemcpy(b->d_small_off, P.small_off.data(), sizeof(int64_t) * b->nsmall,
                                    cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (e = cudaMemcpy(b->d_bp, P.hb.data(), sizeof(BinParams) * nframes, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_atom_off, P.off.data(), sizeof(int64_t) * nframes, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(b->counters, 0, 8 * C_NCOUNTERS)) != cudaSuccess) {
    rs = cuda_fail(ctx, e, "ptm_batch_create");
    batch_free(b);
    return rs;
  }
  *out = b;
  return PTM_OK;
}

extern "C" ptm_status ptm_batch_run(ptm_batch *b, void *stream) {
  if (!b) return PTM_ERR_INVALID_ARG;
  ptm_context *ctx = b->ctx;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (b->exec) {
    CK(cudaGraphLaunch(b->exec, st));
    return PTM_OK;
  }
  return batch_enqueue(b, st);
}

extern "C" ptm_status ptm_batch_capture(ptm_batch *b, void *stream) {
  if (!b || !stream) return PTM_ERR_INVALID_ARG;
  ptm_context *ctx = b->ctx;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  ptm_status rs = batch_enqueue(b, st);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &g);
  if (rs != PTM_OK) { if (g) cudaGraphDestroy(g); return rs; }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
  b->graph = g;
  CK(cudaGraphInstantiate(&b->exec, g, 0));
  return PTM_OK;
}

extern "C" ptm_status ptm_batch_stats(ptm_batch *b, ptm_stats *out) {
  if (!b || !out) return PTM_ERR_INVALID_ARG;
  ptm_context *ctx = b->ctx;
  CK(cudaSetDevice(ctx->device));
  CK(cudaEventSynchronize(b->ev[2]));
  unsigned long long c[C_NCOUNTERS];
  CK(cudaMemcpy(c, b->counters, sizeof c, cudaMemcpyDeviceToHost));
  float t_all = -1.f, t_atom = -1.f;
  if (cudaEventElapsedTime(&t_all, b->ev[0], b->ev[2]) != cudaSuccess) t_all = -1.f;
  if (cudaEventElapsedTime(&t_atom, b->ev[1], b->ev[2]) != cudaSuccess) t_atom = -1.f;
  float t_cls = -1.f, t_match = -1.f;
  if (cudaEventElapsedTime(&t_cls, b->ev[3], b->ev[2]) != cudaSuccess) t_cls = -1.f;
  if (cudaEventElapsedTime(&t_match, b->ev[4], b->ev[2]) != cudaSuccess) t_match = -1.f;
  out->classify_kernel_ms = t_cls;
  out->match_kernel_ms = t_match;
  out->kernel_launches = b->launches;
  cudaGetLastError();
  out->atoms = (int64_t)c[C_ATOMS]; out->matched = (int64_t)c[C_MATCHED]; out->knn_wide = (int64_t)c[C_KNN_WIDE];
  out->knn_fail = (int64_t)c[C_KNN_FAIL]; out->sos = (int64_t)c[C_SOS]; out->qcp_fp64 = (int64_t)c[C_QCP64];
  out->tie_fp64 = (int64_t)c[C_TIE64];
  out->topo_fp64 = (int64_t)c[C_TOPO64]; out->internal = (int64_t)c[C_INTERNAL];
  out->knn_fp64 = (int64_t)c[C_KNN64]; out->excluded = (int64_t)c[C_EXCLUDED];
  out->candidates = (int64_t)c[C_CAND]; out->candidate_points = (int64_t)c[C_CANDPTS];
  out->pipeline_ms = t_all;
  out->atom_kernel_ms = t_atom;
  return PTM_OK;
}

extern "C" ptm_status ptm_batch_destroy(ptm_batch *b) {
  if (!b) return PTM_ERR_INVALID_ARG;
  cudaSetDevice(b->ctx->device);
  for (int i = 0; i < 3; i++) if (b->ev[i]) cudaEventSynchronize(b->ev[i]);
  batch_free(b);
  cudaGetLastError();
  return PTM_OK;
}

// Autotuner: time every (cell size factor, queue tile, blocks per SM) candidate
// on the caller's batch, or on every m-th frame of it when it holds more than
// about 40 M atoms (one warm run, then the best of two timed runs), and return the
// fastest.  Outputs are overwritten with identical results.
extern "C" ptm_status ptm_autotune_batch(ptm_context *ctx, int nframes, const ptm_frame *frames,
                                         const ptm_outputs *outs, void *stream, ptm_tuning *best) {
  if (!ctx || !best) return PTM_ERR_INVALID_ARG;
  static const double factors[] = {1.125, 1.25, 1.4};
  static const int tiles[] = {32, 64};
  static const int bpsm[] = {PTM_ATOM_BLOCKS_PER_SM - 1, PTM_ATOM_BLOCKS_PER_SM};
  cudaStream_t st = (cudaStream_t)stream;
  // tune on every m-th frame so that at most about 40 M atoms are timed per candidate (a
  // strided subset of a mixed batch measured a different winner than the whole)
  int64_t total = 0;
  for (int f = 0; f < nframes; f++) total += frames[f].n_atoms;
  const int64_t cap = 40000000;
  const int stride = (int)std::max<int64_t>(1, (total + cap - 1) / cap);
  std::vector<ptm_frame> fs;
  std::vector<ptm_outputs> os;
  for (int f = 0; f < nframes; f += stride) { fs.push_back(frames[f]); os.push_back(outs[f]); }
  nframes = (int)fs.size();
  frames = fs.data();
  outs = os.data();
  float best_ms = INFINITY;
  for (double fc : factors)
    for (int tl : tiles)
      for (int bs : bpsm) {
        ptm_tuning t = {fc, tl, bs};
        ptm_batch *b = nullptr;
        ptm_status rs = ptm_batch_create(ctx, nframes, frames, outs, &t, &b);
        if (rs != PTM_OK) return rs;
        float ms = INFINITY;
        for (int r = 0; r < 3 && rs == PTM_OK; r++) {
          rs = batch_enqueue(b, st);
          if (rs != PTM_OK) break;
          if (r >= 1) {
            float m = 0.f;
            cudaError_t e = cudaEventSynchronize(b->ev[2]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&m, b->ev[0], b->ev[2]);
            if (e != cudaSuccess) { rs = cuda_fail(ctx, e, "ptm_autotune_batch"); break; }
            ms = std::min(ms, m);
          }
        }
        batch_free(b);
        if (rs != PTM_OK) return rs;
        if (ms < best_ms) { best_ms = ms; *best = t; }
      }
  return PTM_OK;
}

// ============================================================ no-allocation entry
// ptm_classify_frame_noalloc: the same kernels with their workspace in one
// file-scope device array, for callers that cannot allocate device memory.  The
// array is sized for frames of up to PTM_NOALLOC_MAX_ATOMS atoms and stays
// resident on every device that loads the library until the process exits.
namespace {

constexpr int kNoallocAtoms = PTM_NOALLOC_MAX_ATOMS;
constexpr size_t kNoallocCells = max_cells(kNoallocAtoms);          // setup_frame's cap for the largest frame
constexpr size_t kNoallocScanBlocks = (kNoallocCells + 1 + 2 * SCAN_BLOCK - 1) / (2 * SCAN_BLOCK) + 1;

struct NoallocLayout {                  // byte offsets inside the static array
  static constexpr size_t sorted = 0;                                            // Atom64 records (float4 fits too)
  static constexpr size_t sbin = sorted + sizeof(Atom64) * kNoallocAtoms;
  static constexpr size_t wrapv = sbin + sizeof(int) * kNoallocAtoms;
  static constexpr size_t atom_cell = wrapv + sizeof(int) * kNoallocAtoms;
  static constexpr size_t atom_rank = atom_cell + sizeof(int) * kNoallocAtoms;
  static constexpr size_t atom_wrap = atom_rank + sizeof(int) * kNoallocAtoms;
  static constexpr size_t cell_count = atom_wrap + sizeof(int) * kNoallocAtoms;
  static constexpr size_t cell_start = cell_count + sizeof(int) * (kNoallocCells + 1);
  static constexpr size_t block_sums = cell_start + sizeof(int) * (kNoallocCells + 1);
  static constexpr size_t nbr = (block_sums + sizeof(int) * kNoallocScanBlocks + 15) / 16 * 16;
  static constexpr size_t lam = nbr + sizeof(int2) * PTM_KNN * kNoallocAtoms;
  static constexpr size_t ents = lam + sizeof(uint64_t) * 3 * kNoallocAtoms;
  static constexpr size_t tab = (ents + sizeof(uint32_t) * kNoallocAtoms + 15) / 16 * 16;
  static constexpr size_t dstat = tab + sizeof(ShiftTables);
  static constexpr size_t counters = ((dstat + sizeof(int) * 8) + 7) / 8 * 8;
  static constexpr size_t total = counters + sizeof(unsigned long long) * C_NCOUNTERS;
};

static __device__ __align__(256) unsigned char ptm_noalloc_scratch[NoallocLayout::total];

// The array's device address belongs to the CUDA context current when it is
// looked up.  Outside stream capture every call looks it up again (cheap, and
// right after a device reset or with a caller-made driver context); during
// capture, where a lookup may not be allowed, the address found last for the
// current context is used.
typedef int (*CtxGetCurrentFn)(void **);
constexpr int kNoallocCtxSlots = 64;
struct NoallocSlot { void *ctx; unsigned char *ptr; };
NoallocSlot g_noalloc_slots[kNoallocCtxSlots] = {};
int g_noalloc_next = 0;
CtxGetCurrentFn g_ctx_get_current = nullptr;
std::mutex g_noalloc_mutex;

ptm_status noalloc_address(cudaStream_t st, unsigned char **out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_ctx_get_current) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return PTM_ERR_CUDA;
    }
    g_ctx_get_current = (CtxGetCurrentFn)fn;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) { cudaGetLastError(); return PTM_ERR_CUDA; }
  void *ctx = nullptr;
  if (cap == cudaStreamCaptureStatusNone) {
    void *p = nullptr;           // also makes the runtime's context current on a fresh thread
    if (cudaGetSymbolAddress(&p, ptm_noalloc_scratch) != cudaSuccess || !p) { cudaGetLastError(); return PTM_ERR_CUDA; }
    if (g_ctx_get_current(&ctx) != 0 || !ctx) return PTM_ERR_CUDA;
    int k = 0;
    while (k < kNoallocCtxSlots && g_noalloc_slots[k].ctx != ctx) k++;
    if (k == kNoallocCtxSlots) { k = g_noalloc_next; g_noalloc_next = (k + 1) % kNoallocCtxSlots; }
    g_noalloc_slots[k] = {ctx, (unsigned char *)p};
    *out = (unsigned char *)p;
    return PTM_OK;
  }
  if (g_ctx_get_current(&ctx) != 0 || !ctx) return PTM_ERR_CUDA;
  for (int k = 0; k < kNoallocCtxSlots; k++)
    if (g_noalloc_slots[k].ctx == ctx) { *out = g_noalloc_slots[k].ptr; return PTM_OK; }
  return PTM_ERR_INVALID_ARG;    // captured before any call outside capture in this context
}

}  // namespace

extern "C" ptm_status ptm_classify_frame_noalloc(const ptm_frame *f, const ptm_outputs *o, void *stream) {
  if (!f || !o) return PTM_ERR_INVALID_ARG;
  if (f->n_atoms < 1 || f->n_atoms > kNoallocAtoms || !f->positions) return PTM_ERR_INVALID_ARG;
  if (f->ordering != PTM_ORDER_EUCLIDEAN) return PTM_ERR_INVALID_ARG;
  FrameDesc desc;
  BinParams bp;
  ShiftTables tab;
  size_t ncell = 0;
  ptm_status rs = setup_frame(f, 1.25, &desc, &bp, &ncell, &tab);
  if (rs != PTM_OK) return rs;
  if (ncell > kNoallocCells) return PTM_ERR_INVALID_ARG;      // cannot happen: setup_frame caps the grid
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char *base = nullptr;
  rs = noalloc_address(st, &base);
  if (rs != PTM_OK) return rs;
  const int64_t n = f->n_atoms;
  const int f64 = desc.f64;
  void *sorted = base + NoallocLayout::sorted;
  int *sbin = (int *)(base + NoallocLayout::sbin), *wrapv = (int *)(base + NoallocLayout::wrapv);
  int *atom_cell = (int *)(base + NoallocLayout::atom_cell), *atom_rank = (int *)(base + NoallocLayout::atom_rank);
  int *atom_wrap = (int *)(base + NoallocLayout::atom_wrap);
  int *cell_count = (int *)(base + NoallocLayout::cell_count), *cell_start = (int *)(base + NoallocLayout::cell_start);
  int *block_sums = (int *)(base + NoallocLayout::block_sums), *dstat = (int *)(base + NoallocLayout::dstat);
  unsigned long long *counters = (unsigned long long *)(base + NoallocLayout::counters);
  desc.sorted = sorted; desc.sbin = sbin; desc.cell_start = cell_start; desc.wrapv = wrapv;
  desc.nbr = (int2 *)(base + NoallocLayout::nbr);
  desc.lam = (uint64_t *)(base + NoallocLayout::lam);
  desc.ents = (uint32_t *)(base + NoallocLayout::ents);
  desc.tab = (ShiftTables *)(base + NoallocLayout::tab);
  set_outputs(&desc, o);
  desc.dstat = dstat;
  desc.counters = counters;
  bp.counters = counters;
  cudaGetLastError();   // launch errors are read below; drop any left by earlier calls
  // the array keeps the previous call's contents: clear what must start at zero
  if (cudaMemsetAsync(cell_count, 0, (ncell + 1) * sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(dstat, 0, 8 * sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(counters, 0, C_NCOUNTERS * sizeof(unsigned long long), st) != cudaSuccess) {
    cudaGetLastError();
    return PTM_ERR_CUDA;
  }
  k_put_tables<<<1, 256, 0, st>>>(tab, (ShiftTables *)desc.tab);
  const int tb = 256;
  const unsigned gb = (unsigned)((n + tb - 1) / tb);
  k_bin<<<gb, tb, 0, st>>>(f->positions, bp, cell_count, atom_cell, atom_rank, atom_wrap, dstat);
  const int nscan = (int)ncell + 1;
  const int nblk = (nscan + 2 * SCAN_BLOCK - 1) / (2 * SCAN_BLOCK);
  k_scan_block<<<nblk, SCAN_BLOCK, 0, st>>>(cell_count, cell_start, block_sums, nscan);
  k_scan_sums<<<1, SCAN_BLOCK, 0, st>>>(block_sums, nblk, dstat + 2);
  k_scan_add<<<(nscan + 255) / 256, 256, 0, st>>>(cell_start, block_sums, nscan);
  k_scatter<<<gb, tb, 0, st>>>(f->positions, f64, n, atom_cell, atom_rank, atom_wrap, cell_start, sorted, sbin, wrapv);
  const unsigned gk = (unsigned)((n + PTM_KNN_BLOCK - 1) / PTM_KNN_BLOCK);
  if (f64) k_knn<true><<<gk, PTM_KNN_BLOCK, knn_smem_bytes(), st>>>(desc);
  else k_knn<false><<<gk, PTM_KNN_BLOCK, knn_smem_bytes(), st>>>(desc);
  const unsigned ga = (unsigned)((n + PTM_BLOCK - 1) / PTM_BLOCK);
  if (f64) k_hulls<true><<<ga, PTM_BLOCK, atom_smem_bytes(), st>>>(desc);
  else k_hulls<false><<<ga, PTM_BLOCK, atom_smem_bytes(), st>>>(desc);
  if (f64) k_match<true><<<ga, PTM_BLOCK, match_smem_bytes(), st>>>(desc);
  else k_match<false><<<ga, PTM_BLOCK, match_smem_bytes(), st>>>(desc);
  if (cudaGetLastError() != cudaSuccess) return PTM_ERR_CUDA;
  return PTM_OK;
}

// ------------------------------------------------------------ RMSD histogram
// Per-structure histogram of the RMSD of matched atoms (Sec. 5.1: RMSD_max is
// chosen from it).  Each block counts into shared memory, then adds its counts
// to the global array.
namespace ptm {
__global__ void k_rmsd_hist(const int8_t *__restrict__ structure, const float *__restrict__ rmsd, int64_t n,
                            int nbins, float scale, unsigned long long *counts) {
  extern __shared__ unsigned int hs[];            // 5 x (nbins + 1)
  const int nb1 = nbins + 1;
  for (int i = threadIdx.x; i < 5 * nb1; i += blockDim.x) hs[i] = 0u;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int S = structure[i];
    const float r = rmsd[i];
    if (S < 1 || S > 5 || !(r < INFINITY)) continue;          // unmatched
    const int b = min(max((int)floorf(__fmul_rn(r, scale)), 0), nbins);
    atomicAdd(&hs[(S - 1) * nb1 + b], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 5 * nb1; i += blockDim.x)
    if (hs[i]) atomicAdd(&counts[i], (unsigned long long)hs[i]);
}
}  // namespace ptm

extern "C" ptm_status ptm_rmsd_histogram(ptm_context *ctx, int64_t n_atoms, const int8_t *structure, const float *rmsd,
                                         int nbins, double rmsd_max, int64_t *counts, void *stream) {
  using namespace ptm;
  if (!ctx || !structure || !rmsd || !counts || n_atoms < 0 || nbins < 1 || nbins > PTM_HIST_MAX_BINS ||
      !(rmsd_max > 0.0) || !std::isfinite(rmsd_max))
    return PTM_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  cudaGetLastError();
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemsetAsync(counts, 0, sizeof(int64_t) * 5 * (size_t)(nbins + 1), st));
  if (n_atoms == 0) return PTM_OK;
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  const unsigned grid = (unsigned)std::min<int64_t>((n_atoms + 255) / 256, (int64_t)sms * 4);
  const size_t smem = sizeof(unsigned int) * 5 * (size_t)(nbins + 1);
  k_rmsd_hist<<<grid, 256, smem, st>>>(structure, rmsd, n_atoms, nbins, (float)(nbins / rmsd_max),
                                       (unsigned long long *)counts);
  CK(cudaGetLastError());
  return PTM_OK;
}

#include "ptm_serve.cuh"
#include "ptm_peak.cuh"
