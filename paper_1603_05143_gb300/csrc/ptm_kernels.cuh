// Device code of libptm.so: the per-atom classification and the cell-list
// kernels (Larsen, Schmidt & Schiotz, "Robust Structural Identification via
// Polyhedral Template Matching").
//
// Device pipeline for one frame, all on the caller's stream:
//   k_bin      fractional coordinates, cell of each atom (cell list)
//   k_scan_*   exclusive scan of the cell counts
//   k_scatter  atoms copied into cell order as float4 (x, y, z, id)
//   k_knn      one thread per atom: its 14 nearest images, as a neighbour list
//              (k_topo in ptm_topo.cuh instead for the topological order)
//   k_hulls    one thread per atom: hulls, Weinberg codes, template lookup
//   k_match    one thread per atom: QCP, selection, outputs
// The phases run as separate kernels so that the warps of an SM share one
// phase of the method and its code (the instruction cache held none of the
// fused per-atom program).
#pragma once
#include "ptm_atom.cuh"
#include "../../include/ptm.h"

namespace ptm {

template <bool F64> struct RT { typedef float T; };
template <> struct RT<true> { typedef double T; };

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

template <bool F64>
__device__ __forceinline__ void load_atom(const FrameDesc &d, int j, typename RT<F64>::T &x,
                                          typename RT<F64>::T &y, typename RT<F64>::T &z, int &id) {
  if constexpr (F64) {
    const Atom64 *a = (const Atom64 *)d.sorted + j;
    double2 p = __ldg((const double2 *)a);
    double2 q = __ldg((const double2 *)a + 1);
    x = p.x; y = p.y; z = q.x; id = (int)__double_as_longlong(q.y);
  } else {
    float4 p = __ldg((const float4 *)d.sorted + j);
    x = p.x; y = p.y; z = p.z; id = __float_as_int(p.w);
  }
}

// Contract shift of image (a, b, c) in the input precision.
template <bool F64>
__device__ __forceinline__ void contract_shift(const FrameDesc &d, int a, int b, int c, typename RT<F64>::T &sx,
                                               typename RT<F64>::T &sy, typename RT<F64>::T &sz) {
  if constexpr (F64) {
    shift_f64(d, a, b, c, sx, sy, sz);
  } else {
    float lx, ly, lz;
    shift_f32(d, a, b, c, sx, sy, sz, lx, ly, lz);
  }
}

// The distance contract (Sec. 3 orders neighbours by distance; the paper fixes
// no precision, so the order is that of the distances between the given points
// in FP64): dr = (x_j - x_i) + shift, d2 = (dr_x^2 + dr_y^2) + dr_z^2, one
// rounded IEEE operation at a time, no fused multiply-add, float32 positions
// widened exactly.  The kernels first run the same sequence in the input
// precision (FP32 for float32 input) and decide in FP64 only where the FP32
// values cannot order two candidates (knn_err).
__device__ __forceinline__ float contract_dr(float xj, float xi, float s) { return __fadd_rn(__fsub_rn(xj, xi), s); }
__device__ __forceinline__ double contract_dr(double xj, double xi, double s) { return __dadd_rn(__dsub_rn(xj, xi), s); }
__device__ __forceinline__ float contract_d2(float a, float b, float c) {
  return __fadd_rn(__fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b)), __fmul_rn(c, c));
}
__device__ __forceinline__ double contract_d2(double a, double b, double c) {
  return __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
}

// FP64 squared distance of the image (a0, a1, a2) of an atom at (xj, yj, zj):
// the ordering key.  For float64 input it equals the input-precision value.
template <typename T>
__device__ __forceinline__ double key64(const FrameDesc &d, T xj, T yj, T zj, T xi, T yi, T zi, int a0, int a1,
                                        int a2) {
  if constexpr (sizeof(T) == 4) {
    // image 0 with every FP32 difference exact (Sterbenz: |x_j - x_i| <=
    // min(|x_i|, |x_j|)): the FP64 differences are these FP32 values and the
    // zero shift adds nothing, so only the squares and sums run in FP64
    if ((a0 | a1 | a2) == 0) {
      const float px = __fsub_rn(xj, xi), py = __fsub_rn(yj, yi), pz = __fsub_rn(zj, zi);
      if (fabsf(px) <= fminf(fabsf(xi), fabsf(xj)) && fabsf(py) <= fminf(fabsf(yi), fabsf(yj)) &&
          fabsf(pz) <= fminf(fabsf(zi), fabsf(zj)))
        return contract_d2((double)px, (double)py, (double)pz);
    }
  }
  double sx, sy, sz;
  shift_f64(d, a0, a1, a2, sx, sy, sz);
  return contract_d2(contract_dr((double)xj, (double)xi, sx), contract_dr((double)yj, (double)yi, sy),
                     contract_dr((double)zj, (double)zi, sz));
}

// Bound on |d2_32 - d2_64| for an FP32 contract value v whose image shift has
// length at most S (u = 2^-24).  Each component of the FP32 vector is within
// 2u (|dr_c| + |s_c|) of the FP64 one (the difference, the shift's rounding to
// FP32 and the sum each round once); squaring and the two sums add 3u v.  So
// |d2_32 - d2_64| <= u (7 v + 4 |dr| |s|) + 8 u^2 (v + S^2); the constants
// below leave room for |dr| estimated from v and for rounding in this bound.
__device__ __forceinline__ float knn_err(float v, float S) {
  const float u = 5.9604645e-8f;
  return u * (8.5f * v + 4.5f * sqrtf(v) * S + 9.f * u * S * S);
}

// Key order (FP64 d2, atom id, image).  Keys are non-negative and not NaN, so
// their bit patterns order as unsigned integers: the comparisons stay off the
// FP64 pipe.
__device__ __forceinline__ bool key_less64(double da, int ia, int ma, double db, int ib, int mb) {
  const unsigned long long ua = (unsigned long long)__double_as_longlong(da);
  const unsigned long long ub = (unsigned long long)__double_as_longlong(db);
  return ua < ub || (ua == ub && (ia < ib || (ia == ib && ma < mb)));
}

// ----------------------------------------------------------------- kNN
// Visit every (atom, image) in the (2R+1)^3 cells around cell (bx, by, bz):
// visit(j, d2, idj, a0, a1, a2, xj, yj, zj, sx, sy, sz) with d2 by the contract
// in the input precision, (a0, a1, a2) the image and (sx, sy, sz) its shift.
// The cells bz - R .. bz + R of a column are consecutive in the sorted order
// unless the range wraps, and are then scanned as one range of atoms.
template <bool F64, typename V>
__device__ __forceinline__ void scan_cells(const FrameDesc &d, int s, typename RT<F64>::T xi,
                                           typename RT<F64>::T yi, typename RT<F64>::T zi, int bx, int by, int bz,
                                           int wix, int wiy, int wiz, bool wrapped, int R, V &&visit) {
  typedef typename RT<F64>::T T;
  const int nbx = d.nb[0], nby = d.nb[1], nbz = d.nb[2];
  for (int ix = 0; ix <= 2 * R; ix++) {
    const int dx = ix <= R ? ix : R - ix;                // 0, 1 .. R, -1 .. -R: the centre first
    int cx = bx + dx, mx = 0;
    if (d.pbc[0]) { mx = floordiv(cx, nbx); cx -= mx * nbx; } else if (cx < 0 || cx >= nbx) continue;
    for (int iy = 0; iy <= 2 * R; iy++) {
      const int dy = iy <= R ? iy : R - iy;
      int cy = by + dy, my = 0;
      if (d.pbc[1]) { my = floordiv(cy, nby); cy -= my * nby; } else if (cy < 0 || cy >= nby) continue;
      int z0 = bz - R, z1 = bz + R;
      if (!d.pbc[2]) { z0 = max(z0, 0); z1 = min(z1, nbz - 1); }
      const bool column = z0 >= 0 && z1 < nbz;             // no wrap: one range, image mz = 0
      const int cbase = (cx * nby + cy) * nbz;
      for (int r = 0; r < (column ? 1 : 2 * R + 1); r++) {
        int ca = cbase + z0, cb = cbase + z1, mz = 0;     // cells ca .. cb
        if (!column) {
          int cz = bz - R + r;
          mz = floordiv(cz, nbz);                          // periodic z (else column)
          cz -= mz * nbz;
          ca = cb = cbase + cz;
        }
        const int j0 = __ldg(d.cell_start + ca), j1 = __ldg(d.cell_start + cb + 1);
        if (j0 == j1) continue;
        const int n0 = mx + wix, n1 = my + wiy, n2 = mz + wiz;
        T sx, sy, sz;
        contract_shift<F64>(d, n0, n1, n2, sx, sy, sz);
#pragma unroll 2
        for (int j = j0; j < j1; j++) {
          T xj, yj, zj;
          int idj;
          load_atom<F64>(d, j, xj, yj, zj, idj);
          int a0 = n0, a1 = n1, a2 = n2;
          if (wrapped) {
            int w0, w1, w2;
            img_unpack(__ldg(d.wrapv + j), w0, w1, w2);
            a0 -= w0; a1 -= w1; a2 -= w2;
            contract_shift<F64>(d, a0, a1, a2, sx, sy, sz);
          }
          if (j == s && a0 == 0 && a1 == 0 && a2 == 0) continue;
          const T ex = contract_dr(xj, xi, sx), ey = contract_dr(yj, yi, sy), ez = contract_dr(zj, zi, sz);
          visit(j, contract_d2(ex, ey, ez), idj, a0, a1, a2, xj, yj, zj, sx, sy, sz);
        }
      }
    }
  }
}

__device__ __forceinline__ bool search_complete(const FrameDesc &d, int R, float d2_last) {
  const float rg = (float)R * d.min_cell_width - __int_as_float(d.dstat[1]);
  return rg > 0.f && d2_last < rg * rg * (1.f - 1e-3f);
}

// General kNN: the NK nearest images of atom s by the full key (FP64 d2, atom
// id, image), R growing until the NK-th distance lies inside the radius the
// scanned cells are guaranteed to cover.  For float32 input a candidate whose
// FP32 distance, less its error bound, exceeds the current NK-th key cannot
// enter and skips the FP64 evaluation.  Returns the neighbour count (NK, fewer
// only for a small fully non-periodic system) or -1.
template <bool F64, int NK = PTM_KNN>
__device__ __noinline__ int knn(const FrameDesc &d, int s, typename RT<F64>::T xi, typename RT<F64>::T yi,
                                typename RT<F64>::T zi, int bx, int by, int bz, int wix, int wiy, int wiz,
                                bool wrapped, double (&Ld2)[NK], int (&Lid)[NK], int (&Ljs)[NK], int (&Limg)[NK]) {
  typedef typename RT<F64>::T T;
  for (int R = 1; R <= PTM_RMAX; R++) {
    float last32 = INFINITY;                           // the NK-th key rounded up to FP32
#pragma unroll
    for (int t = 0; t < NK; t++) { Ld2[t] = INFINITY; Lid[t] = 0x7fffffff; Ljs[t] = -1; Limg[t] = 0x7fffffff; }
    scan_cells<F64>(d, s, xi, yi, zi, bx, by, bz, wix, wiy, wiz, wrapped, R,
                    [&](int j, T d2, int idj, int a0, int a1, int a2, T xj, T yj, T zj, T sx, T sy, T sz) {
      double key;
      if constexpr (F64) {
        key = d2;
      } else {
        const float S = sqrtf(sx * sx + sy * sy + sz * sz) * 1.0001f;
        if (d2 - 1.25f * knn_err(d2, S) > last32) return;
        key = key64(d, xj, yj, zj, xi, yi, zi, a0, a1, a2);
      }
      if ((unsigned long long)__double_as_longlong(key) > (unsigned long long)__double_as_longlong(Ld2[NK - 1])) return;
      const int img = img_pack(a0, a1, a2);
      if (!key_less64(key, idj, img, Ld2[NK - 1], Lid[NK - 1], Limg[NK - 1])) return;
      // insertion into the sorted list (all indices static: stays in registers)
      bool above = true;
#pragma unroll
      for (int t = NK - 1; t >= 1; t--) {
        bool lt = key_less64(key, idj, img, Ld2[t - 1], Lid[t - 1], Limg[t - 1]);
        if (lt) { Ld2[t] = Ld2[t - 1]; Lid[t] = Lid[t - 1]; Ljs[t] = Ljs[t - 1]; Limg[t] = Limg[t - 1]; }
        else if (above) { Ld2[t] = key; Lid[t] = idj; Ljs[t] = j; Limg[t] = img; }
        above = lt;
      }
      if (above) { Ld2[0] = key; Lid[0] = idj; Ljs[0] = j; Limg[0] = img; }
      if constexpr (!F64) last32 = __double2float_ru(Ld2[NK - 1]);
    });
    if (search_complete(d, R, __double2float_ru(Ld2[NK - 1]))) {
      if (R > 1) count(d, C_KNN_WIDE);
      return NK;
    }
    if (!d.pbc[0] && !d.pbc[1] && !d.pbc[2] && R >= max(d.nb[0], max(d.nb[1], d.nb[2]))) {
      int cnt = 0;
#pragma unroll
      for (int t = 0; t < NK; t++) cnt += Ljs[t] >= 0;
      return cnt;
    }
  }
  count(d, C_KNN_FAIL);
  return -1;
}

// Fast kNN for the common case (27 cells suffice).  Pass 1 keeps the NK + 1
// smallest distances in the input precision with a min/max network.  Slots t
// and t + 1 are "close" when those values could order their candidates
// differently from FP64 (float32 input: the gap is within twice knn_err;
// float64 input: equal values); close slots form runs, and the last run also
// takes every candidate beyond slot NK - 1 within the error band.  Pass 2
// rescans and drops each candidate into its rank slot; a run's candidates are
// placed by insertion on the full key (FP64 d2, atom id, image), keeping the
// smallest keys when the run crosses the last slot, so the result is the
// general kNN's order.  Slots are written through `rows`: put(r, j, img) and,
// inside runs, set(r, j, img, id, key) / j(r) / img(r) / id(r) / key(r)
// (j = -1: empty).  `close_runs` receives the run mask (0: every rank decided
// in the input precision).  Returns false when the general kNN must decide.
template <bool F64, int NK, typename Rows>
__device__ __forceinline__ bool knn_fast_n(const FrameDesc &d, int s, typename RT<F64>::T xi,
                                           typename RT<F64>::T yi, typename RT<F64>::T zi, int bx, int by, int bz,
                                           const Rows &rows, uint32_t &close_runs) {
  typedef typename RT<F64>::T T;
  // float32 input, 14 neighbours: the network also carries each value's
  // candidate as (sorted slot << 5 | image index), so that an atom whose ranks
  // are all decided needs no second scan (slots below 2^27)
  constexpr bool CARRY = !F64 && NK == PTM_KNN;
  T L[NK + 1];
  uint32_t C[CARRY ? NK + 1 : 1];
#pragma unroll
  for (int t = 0; t <= NK; t++) L[t] = (T)INFINITY;
  if constexpr (CARRY) {
#pragma unroll
    for (int t = 0; t <= NK; t++) C[t] = 0u;
  }
  scan_cells<F64>(d, s, xi, yi, zi, bx, by, bz, 0, 0, 0, false, 1,
                  [&](int j, T d2, int, int a0, int a1, int a2, T, T, T, T, T, T) {
    if (!(d2 < L[NK])) return;
    T x = d2;
    if constexpr (CARRY) {
      uint32_t xc = ((uint32_t)j << 5) | (uint32_t)((a0 + 1) * 9 + (a1 + 1) * 3 + (a2 + 1));
#pragma unroll
      for (int t = 0; t <= NK; t++) {
        const bool sw = x < L[t];
        const T lo = sw ? x : L[t];
        const uint32_t lc = sw ? xc : C[t];
        x = sw ? L[t] : x;
        xc = sw ? C[t] : xc;
        L[t] = lo;
        C[t] = lc;
      }
    } else {
#pragma unroll
      for (int t = 0; t <= NK; t++) { const T lo = fmin(L[t], x); x = fmax(L[t], x); L[t] = lo; }
    }
  });
  if (!(L[NK] < (T)INFINITY)) return false;
  uint32_t close = 0;                                // bit t: slots t and t + 1 in one run
  T limit = L[NK - 1];                               // pass 2 admits d2 <= limit
  if constexpr (F64) {
#pragma unroll
    for (int t = 0; t < NK; t++) close |= (uint32_t)(L[t] == L[t + 1]) << t;
  } else {
    // image shifts occur only when the 27 cells wrap around a periodic side
    const bool shifted = (d.pbc[0] && (bx == 0 || bx >= d.nb[0] - 1)) ||
                         (d.pbc[1] && (by == 0 || by >= d.nb[1] - 1)) ||
                         (d.pbc[2] && (bz == 0 || bz >= d.nb[2] - 1));
    // one band for every gap: twice the bound at the largest kept value
    // (knn_err grows with v), without the shift term for an unshifted atom
    const float vmax = 1.01f * L[NK];
    const float band = shifted ? 2.f * knn_err(vmax, d.smax) : 2.f * 8.5f * 5.9604645e-8f * vmax;
#pragma unroll
    for (int t = 0; t < NK; t++) close |= (uint32_t)(L[t + 1] - L[t] <= band) << t;
    if (close >> (NK - 1) & 1) limit = L[NK - 1] + band;
  }
  if (!search_complete(d, 1, (float)limit)) return false;
  close_runs = close;
  if constexpr (CARRY) {
    if (!close && d.atom_offset + d.n <= (1ll << 27)) {    // every rank decided, the candidates at hand
#pragma unroll
      for (int t = 0; t < NK; t++) {
        const int k = (int)(C[t] & 31u);
        rows.put(t, (int)(C[t] >> 5), img_pack(k / 9 - 1, (k / 3) % 3 - 1, k % 3 - 1));
      }
      return true;
    }
  }
  if (!close) {                                      // every rank decided: distance order is key order
    scan_cells<F64>(d, s, xi, yi, zi, bx, by, bz, 0, 0, 0, false, 1,
                    [&](int j, T d2, int, int a0, int a1, int a2, T, T, T, T, T, T) {
      if (!(d2 <= limit)) return;
      int rank = 0;
#pragma unroll
      for (int t = 0; t < NK - 1; t++) rank += L[t] < d2;
      rows.put(rank, j, img_pack(a0, a1, a2));
    });
    return true;
  }
  const bool crossing = (close >> (NK - 1)) & 1;
  for (int r = 0; r < NK; r++) rows.set(r, -1, 0, 0, 0.0);
  scan_cells<F64>(d, s, xi, yi, zi, bx, by, bz, 0, 0, 0, false, 1,
                  [&](int j, T d2, int idj, int a0, int a1, int a2, T xj, T yj, T zj, T, T, T) {
    if (!(d2 <= limit)) return;
    int r0 = 0;                                      // first slot holding this value (NK - 1 beyond)
#pragma unroll
    for (int t = 0; t < NK - 1; t++) r0 += L[t] < d2;
    const uint32_t below = ~close & ((1u << r0) - 1u);
    const int rs = below ? 32 - __clz(below) : 0;    // the run: slots rs .. hi - 1
    const int hi = min(r0 + __ffs(~(close >> r0)), NK);
    const int img = img_pack(a0, a1, a2);
    if (hi - rs == 1 && !(hi == NK && crossing)) { rows.put(rs, j, img); return; }
    double key;
    if constexpr (F64) key = d2;
    else key = key64(d, xj, yj, zj, xi, yi, zi, a0, a1, a2);
    int r = rs;                                      // insertion point by (key, id, image)
    while (r < hi && rows.j(r) >= 0 && key_less64(rows.key(r), rows.id(r), rows.img(r), key, idj, img)) r++;
    if (r == hi) return;                             // beyond the NK nearest
    int e = r;                                       // first empty slot, or the run's last
    while (e < hi - 1 && rows.j(e) >= 0) e++;
    for (int q = e; q > r; q--) rows.set(q, rows.j(q - 1), rows.img(q - 1), rows.id(q - 1), rows.key(q - 1));
    rows.set(r, j, img, idj, key);
  });
  return true;
}

// kNN slots in per-thread shared-memory rows ([row][thread], stride B): row r
// the sorted slot, row NK + r the packed image; while a run is ordered, row
// 2 NK + r the atom id and rows 3 NK + 2 r, 3 NK + 2 r + 1 the FP64 key.
template <int NK, int B>
struct SmemKnnRows {
  int *base;
  int t;
  static constexpr int kRows = 5 * NK;
  __device__ __forceinline__ int &row(int k) const { return base[k * B + t]; }
  __device__ __forceinline__ void put(int r, int j, int img) const {
    row(r) = j;
    row(NK + r) = img;
  }
  __device__ __forceinline__ void set(int r, int j, int img, int id, double key) const {
    put(r, j, img);
    row(2 * NK + r) = id;
    row(3 * NK + 2 * r) = __double2hiint(key);
    row(3 * NK + 2 * r + 1) = __double2loint(key);
  }
  __device__ __forceinline__ int j(int r) const { return row(r); }
  __device__ __forceinline__ int img(int r) const { return row(NK + r); }
  __device__ __forceinline__ int id(int r) const { return row(2 * NK + r); }
  __device__ __forceinline__ double key(int r) const {
    return __hiloint2double(row(3 * NK + 2 * r), row(3 * NK + 2 * r + 1));
  }
};

#define PTM_KNN_BLOCK 128
// 6 blocks of 128 threads per SM: the shared-memory rows (280 B per thread) and
// at most 85 registers per thread fit
#define PTM_KNN_BLOCKS_PER_SM 6
// The batch form (frame lookup per slot, descriptors in global memory) spills
// at 85 registers; at 5 blocks per SM it keeps 96 (batch of 256 frames: 30.4 ->
// 28.5 ms, while the single-frame kernel is faster at 6: 0.824 against 0.864 ms)
#define PTM_KNN_BATCH_BLOCKS_PER_SM 5
typedef SmemKnnRows<PTM_KNN, PTM_KNN_BLOCK> KnnRows;
constexpr size_t knn_smem_bytes() { return (size_t)PTM_KNN_BLOCK * KnnRows::kRows * 4; }

// The 14 nearest images of the atom at sorted slot s (Sec. 3, Table 1), written
// to its neighbour list: fast search when 27 cells suffice, else the general
// one.  A search that fails leaves an empty list (the atom stays unmatched).
template <bool F64>
__device__ __forceinline__ void knn_atom(const FrameDesc &d, int s, int *smem_rows) {
  typedef typename RT<F64>::T T;
  T xi, yi, zi;
  int idi;
  load_atom<F64>(d, s, xi, yi, zi, idi);
  const int b = __ldg(d.sbin + s);
  const int bz = b % d.nb[2], byx = b / d.nb[2];
  const int by = byx % d.nb[1], bx = byx / d.nb[1];
  const bool wrapped = d.dstat[0] != 0;
  const KnnRows rows{smem_rows, (int)threadIdx.x};
  int2 *out = const_cast<int2 *>(d.nbr) + (s - d.atom_offset);
  if (__ldg(d.wrapv + s) == PTM_EXCLUDED) {           // excluded by the binning: no neighbours
#pragma unroll
    for (int t = 0; t < PTM_KNN; t++) out[(int64_t)t * d.n] = make_int2(-1, 0);
    return;
  }
  uint32_t close = 0;
  if (!wrapped && knn_fast_n<F64, PTM_KNN>(d, s, xi, yi, zi, bx, by, bz, rows, close)) {
    if (!F64 && close) count(d, C_KNN64);
#pragma unroll
    for (int t = 0; t < PTM_KNN; t++) out[(int64_t)t * d.n] = make_int2(rows.j(t), rows.img(t));
    return;
  }
  int wix = 0, wiy = 0, wiz = 0;
  if (wrapped) img_unpack(__ldg(d.wrapv + s), wix, wiy, wiz);
  double Ld2[PTM_KNN];
  int Lid[PTM_KNN], Ljs[PTM_KNN], Limg[PTM_KNN];
  const int cnt = knn<F64>(d, s, xi, yi, zi, bx, by, bz, wix, wiy, wiz, wrapped, Ld2, Lid, Ljs, Limg);
  if (!F64) count(d, C_KNN64);
#pragma unroll
  for (int t = 0; t < PTM_KNN; t++) out[(int64_t)t * d.n] = t < cnt ? make_int2(Ljs[t], Limg[t]) : make_int2(-1, 0);
}

// ---------------------------------------------------------- per-atom state
// Per-atom selection state.  Plain scalars (no arrays) so that it stays in
// registers; snapshot k = 6, 12, 14 keeps its walk labelling and table entry.
struct Best {
  float b1, b2;                 // best and second-best FP32 RMSD^2
  int K, cand;                  // winning snapshot (6, 12, 14) and candidate index
  int fp64;                     // the winner's eigenvalue needed the FP64 solve
  uint64_t lam6, lam12, lam14;  // walk labelling per snapshot
  int ent6, ent12, ent14;       // table entry per snapshot, -1 = none
  __device__ __forceinline__ uint64_t lam(int K) const { return K == 6 ? lam6 : (K == 12 ? lam12 : lam14); }
  __device__ __forceinline__ int ent(int K) const { return K == 6 ? ent6 : (K == 12 ? ent12 : ent14); }
};

__device__ __forceinline__ int snap_index(int K) { return K == 6 ? 0 : (K == 12 ? 1 : 2); }

__device__ __forceinline__ int lookup(const Scratch &sm, int K, uint64_t h) {
  const int LEN = 2 * (3 * K - 6) + 1;
  const int NW = (LEN - 2 + 7) / 8;                 // stored labels 3..LEN
  int pos = (int)(h & (PTM_TBL_NSLOTS - 1));
  for (int probe = 0; probe < PTM_TBL_NSLOTS; probe++) {
    const ptm_tbl_entry *e = &ptm_tbl[pos];
    uint64_t eh = __ldg((const unsigned long long *)&e->hash);
    int cntv = __ldg(&e->count);
    if (eh == 0 && cntv == 0) return -1;
    if (eh == h && __ldg(&e->nv) == K) {
      bool eq = true;
#pragma unroll
      for (int w = 0; w < PTM_CODE_WORDS; w++) if (w < NW) eq &= (__ldg(&e->code[w]) == sm.CODE(w));
      if (eq) return pos;
    }
    pos = (pos + 1) & (PTM_TBL_NSLOTS - 1);
  }
  return -1;
}

// S_ab = sum_j w_{slot(j), a} dr_{j, b} for the correspondence "neighbour rank j ->
// template slot" given by the walk labelling and the table candidate.
// Because the template barycentre is the origin and slot 0 (the centre) sits at
// it, the data barycentre drops out of S.
__device__ __forceinline__ void cov_matrix(int K, const Scratch &sm, const float4 *tplw, int S, uint64_t lab,
                                           uint64_t cand, float (&Sm)[3][3]) {
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) Sm[a][b] = 0.f;
#pragma unroll 1
  for (int j = 0; j < K; j++) {
    const int slot = nib(cand, nib(lab, j) - 1);
    const float4 w = __ldg(tplw + S * 15 + slot);
    const float x = sm.DX(j), y = sm.DY(j), z = sm.DZ(j);
    Sm[0][0] = fmaf(w.x, x, Sm[0][0]); Sm[0][1] = fmaf(w.x, y, Sm[0][1]); Sm[0][2] = fmaf(w.x, z, Sm[0][2]);
    Sm[1][0] = fmaf(w.y, x, Sm[1][0]); Sm[1][1] = fmaf(w.y, y, Sm[1][1]); Sm[1][2] = fmaf(w.y, z, Sm[1][2]);
    Sm[2][0] = fmaf(w.z, x, Sm[2][0]); Sm[2][1] = fmaf(w.z, y, Sm[2][1]); Sm[2][2] = fmaf(w.z, z, Sm[2][2]);
  }
}

// Barycentre of the centre and its first K neighbours, and G_v = sum |v - mean|^2.
__device__ __forceinline__ void data_moments(int K, const Scratch &sm, float &mx, float &my, float &mz, float &Gv) {
  float sx = 0, sy = 0, sz = 0, g = 0;
#pragma unroll 1
  for (int j = 0; j < K; j++) {
    const float x = sm.DX(j), y = sm.DY(j), z = sm.DZ(j);
    sx += x; sy += y; sz += z;
    g = fmaf(x, x, fmaf(y, y, fmaf(z, z, g)));
  }
  const float inv = 1.f / (float)(K + 1);
  mx = sx * inv; my = sy * inv; mz = sz * inv;
  Gv = g - (float)(K + 1) * (mx * mx + my * my + mz * mz);
}

// RMSD^2 of one candidate from its covariance (closed form after Eq. 3); the
// FP32 Newton solution is replaced by an FP64 one when the top eigenvalue is
// not well separated (normalised P'(lambda_1) below PTM_GAP).
__device__ __noinline__ float r2_fp64(float s00, float s01, float s02, float s10, float s11, float s12, float s20,
                                      float s21, float s22, float Gv, float Gw, int N) {
  double S[3][3] = {{s00, s01, s02}, {s10, s11, s12}, {s20, s21, s22}};
  Qcp<double> o;
  qcp_solve<double>(S, (double)Gv, (double)Gw, o);
  return (float)(((double)Gw - o.lam * o.lam / (double)Gv) / N);
}

__device__ __forceinline__ float cand_r2(const float (&Sm)[3][3], float Gv, float Gw, int N, int &fp64,
                                         const FrameDesc &d) {
  Qcp<float> o;
  qcp_solve<float>(Sm, Gv, Gw, o);
  float B = sqrtf(Gv * Gw);
  float gamma = o.dP / (B * B * B);
  if (!(gamma >= PTM_GAP) || o.iters >= 60) {
    fp64 = 1;
    count(d, C_QCP64);
    return fmaxf(r2_fp64(Sm[0][0], Sm[0][1], Sm[0][2], Sm[1][0], Sm[1][1], Sm[1][2], Sm[2][0], Sm[2][1], Sm[2][2],
                         Gv, Gw, N), 0.f);
  }
  fp64 = 0;
  return fmaxf((Gw - o.lam * o.lam / Gv) / (float)N, 0.f);
}

// Hull of the first K neighbours is complete and contains the centre: Weinberg
// code and lookup (Algorithm 1, inner loops).  Only the labelling and table
// entry are kept; every snapshot's candidates are scored after the last one, in
// one loop (score_candidates, or select_fp64 in the FP64 form).
__device__ void snapshot(int K, const Scratch &sm, const FrameDesc &d, int nf, Best &bst) {
  if (nf != 2 * K - 4) return;                    // a neighbour is not a hull vertex
  uint64_t lab = 0, h = 0;
  if (!canonical(sm, K, nf, lab, h, d)) return;
  int e = lookup(sm, K, h);
  if (e < 0) return;
  if (K == 6) { bst.lam6 = lab; bst.ent6 = e; }
  else if (K == 12) { bst.lam12 = lab; bst.ent12 = e; }
  else { bst.lam14 = lab; bst.ent14 = e; }
}

// FP32 QCP of every admissible correspondence of the matched snapshots, in
// snapshot order (6, 12, 14) and table order, as one flat loop whose trips
// start warp-converged (every lane in `qmask` calls it), so the lanes of a warp
// run their candidates together; keeps the best and second-best RMSD^2 (the
// first of equal values wins, Algorithm 1).
__device__ void score_candidates(const FrameDesc &d, const Scratch &sm, const float4 *tplw, Best &bst,
                                 unsigned qmask) {
  int n6 = 0, n12 = 0, n14 = 0, f6 = 0, f12 = 0, f14 = 0;
  float Gv6 = 0.f, Gv12 = 0.f, Gv14 = 0.f, mx, my, mz;
  if (bst.ent6 >= 0) { f6 = ptm_tbl[bst.ent6].first; n6 = ptm_tbl[bst.ent6].count; data_moments(6, sm, mx, my, mz, Gv6); }
  if (bst.ent12 >= 0) { f12 = ptm_tbl[bst.ent12].first; n12 = ptm_tbl[bst.ent12].count; data_moments(12, sm, mx, my, mz, Gv12); }
  if (bst.ent14 >= 0) { f14 = ptm_tbl[bst.ent14].first; n14 = ptm_tbl[bst.ent14].count; data_moments(14, sm, mx, my, mz, Gv14); }
  const int total = n6 + n12 + n14;
  int scored = 0, points = 0;
  for (int i = 0; __any_sync(qmask, i < total); i++) {
    if (i >= total) continue;
    int K, c;
    uint64_t lab;
    float Gv;
    if (i < n6) { K = 6; c = f6 + i; lab = bst.lam6; Gv = Gv6; }
    else if (i < n6 + n12) { K = 12; c = f12 + (i - n6); lab = bst.lam12; Gv = Gv12; }
    else { K = 14; c = f14 + (i - n6 - n12); lab = bst.lam14; Gv = Gv14; }
    const uint64_t cand = __ldg((const unsigned long long *)&ptm_cand[c]);
    const int S = (int)(cand >> 60) & 7;
    if (!(d.mask >> S & 1)) continue;
    scored++;
    points += K + 1;
    float Sm[3][3];
    cov_matrix(K, sm, tplw, S, lab, cand, Sm);
    const float Gw = __ldg(tplw + S * 15).w;
    int fp64;
    const float r2 = cand_r2(Sm, Gv, Gw, K + 1, fp64, d);
    if (r2 < bst.b1) { bst.b2 = bst.b1; bst.b1 = r2; bst.K = K; bst.cand = c; bst.fp64 = fp64; }
    else if (r2 < bst.b2) bst.b2 = r2;
  }
  if (scored) { count(d, C_CAND, scored); count(d, C_CANDPTS, (unsigned long long)points); }
}

// Canonical correspondence: the paper leaves open which of the equivalent
// correspondences of a match is reported; this library reports the smallest
// member of its orbit under the template's rotation group.  Nibble 15 - s holds
// the neighbour rank of template slot s, so the orbit minimum, read slot 1
// first, is the numerically smallest packing.
__device__ uint64_t canonical_corr(int S, int K, uint64_t corr) {
  uint64_t best = ~0ull;
  const int g0 = ptm_group_off[S], g1 = ptm_group_off[S + 1];
  for (int g = g0; g < g1; g++) {
    uint64_t cur = 0;
    for (int s = 1; s <= K; s++) cur |= (uint64_t)nib(corr, 15 - ptm_group_perm[g][s]) << (4 * (15 - s));
    best = cur < best ? cur : best;
  }
  return best;
}

__device__ __forceinline__ uint64_t corr_of(int K, uint64_t lab, uint64_t cand) {
  uint64_t corr = 0;
#pragma unroll
  for (int j = 0; j < PTM_KNN; j++) {
    if (j >= K) break;
    int slot = nib(cand, nib(lab, j) - 1);
    corr |= (uint64_t)(j + 1) << (4 * (15 - slot));
  }
  return corr;
}


// FP64 selection over every candidate of the matched snapshots (Algorithm 1,
// inner loops), from FP64 neighbour vectors.  Exact ties, which the paper does
// not resolve, are read as: RMSD^2 within PTM_TIE goes to the earlier template
// (SC, FCC, HCP, ICO, BCC), then to the smaller canonical correspondence.
// Returns (K << 16) | candidate index, or -1; *scored counts the candidates.
__device__ __noinline__ int select_fp64(const FrameDesc &d, const Best &bst, const double (&ex)[PTM_KNN],
                                        const double (&ey)[PTM_KNN], const double (&ez)[PTM_KNN], int *scored) {
  double best_r2 = INFINITY;
  int bK = -1, bc = -1, bS = 99, ns = 0;
  uint64_t bcp = ~0ull;
  // pass 0 finds the minimum, pass 1 picks among the candidates tied with it
  for (int pass = 0; pass < 2; pass++) {
    for (int si = 0; si < 3; si++) {
      const int K = si == 0 ? 6 : (si == 1 ? 12 : 14);
      int e = bst.ent(K);
      if (e < 0) continue;
      uint64_t lab = bst.lam(K);
      double m[3] = {0, 0, 0}, g = 0;
      for (int j = 0; j < K; j++) { m[0] += ex[j]; m[1] += ey[j]; m[2] += ez[j]; g += ex[j] * ex[j] + ey[j] * ey[j] + ez[j] * ez[j]; }
      for (int c = 0; c < 3; c++) m[c] /= (K + 1);
      double Gv = g - (K + 1) * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
      const int first = ptm_tbl[e].first, ncand = ptm_tbl[e].count;
      for (int ci = first; ci < first + ncand; ci++) {
        uint64_t cand = ptm_cand[ci];
        int S = (int)(cand >> 60) & 7;
        if (!(d.mask >> S & 1)) continue;
        if (pass == 0) ns++;
        double Sm[3][3] = {{0}}, Gw = 0;
        for (int j = 0; j < K; j++) {
          int slot = nib(cand, nib(lab, j) - 1);
          const double *w = ptm_tpl64[S][slot];
          Sm[0][0] += w[0] * ex[j]; Sm[0][1] += w[0] * ey[j]; Sm[0][2] += w[0] * ez[j];
          Sm[1][0] += w[1] * ex[j]; Sm[1][1] += w[1] * ey[j]; Sm[1][2] += w[1] * ez[j];
          Sm[2][0] += w[2] * ex[j]; Sm[2][1] += w[2] * ey[j]; Sm[2][2] += w[2] * ez[j];
        }
        for (int slot = 0; slot <= K; slot++)
          Gw += ptm_tpl64[S][slot][0] * ptm_tpl64[S][slot][0] + ptm_tpl64[S][slot][1] * ptm_tpl64[S][slot][1] +
                ptm_tpl64[S][slot][2] * ptm_tpl64[S][slot][2];
        Qcp<double> o;
        qcp_solve<double>(Sm, Gv, Gw, o);
        double r2 = fmax((Gw - o.lam * o.lam / Gv) / (K + 1), 0.0);
        if (pass == 0) {
          best_r2 = fmin(best_r2, r2);
        } else if (r2 <= best_r2 + PTM_TIE) {
          uint64_t cp = canonical_corr(S, K, corr_of(K, lab, cand));
          if (S < bS || (S == bS && cp < bcp)) { bS = S; bcp = cp; bK = K; bc = ci; }
        }
      }
    }
  }
  if (scored) *scored = ns;
  return bK > 0 ? (bK << 16) | bc : -1;
}

// FP64 neighbour vector of neighbour (sorted slot js, image img) of an atom at
// (xi, yi, zi): (x_j - x_i) + n.H with the shift exactly as the contract rounds it.
template <bool F64>
__device__ __forceinline__ void vec_fp64(const FrameDesc &d, typename RT<F64>::T xi, typename RT<F64>::T yi,
                                         typename RT<F64>::T zi, int js, int img, double &x, double &y, double &z) {
  typedef typename RT<F64>::T T;
  T xj, yj, zj;
  int idj;
  load_atom<F64>(d, js, xj, yj, zj, idj);
  int a, b, c;
  img_unpack(img, a, b, c);
  double sx, sy, sz;
  shift_f64(d, a, b, c, sx, sy, sz);
  x = ((double)xj - (double)xi) + sx;
  y = ((double)yj - (double)yi) + sy;
  z = ((double)zj - (double)zi) + sz;
}

// Rare path: the best FP32 candidates lie within PTM_BAND.  Every candidate is
// re-scored in FP64 from neighbour vectors recomputed in FP64 from the input
// positions (the neighbours read again from the atom's list).
template <bool F64>
__device__ __noinline__ int rerank_fp64(const FrameDesc &d, int s, const Best bst) {
  typedef typename RT<F64>::T T;
  T xi, yi, zi;
  int idi;
  load_atom<F64>(d, s, xi, yi, zi, idi);
  double ex[PTM_KNN], ey[PTM_KNN], ez[PTM_KNN];
  int cnt = 0;
  for (int t = 0; t < PTM_KNN; t++) {
    const int2 e = d.nbr[(int64_t)t * d.n + (s - d.atom_offset)];
    if (e.x < 0) break;
    vec_fp64<F64>(d, xi, yi, zi, e.x, e.y, ex[t], ey[t], ez[t]);
    cnt++;
  }
  if (cnt == 0) return -1;
  return select_fp64(d, bst, ex, ey, ez, nullptr);
}

// ------------------------------------------------------------ finalisation
// Binary alloy label (Sec. 6, Table 3) of atom a matched to template S with
// canonical correspondence cp (nibble 15 - slot = neighbour rank + 1).
__device__ __forceinline__ int8_t alloy_label(const FrameDesc &d, const Scratch &sm, int S, uint64_t cp, int64_t a) {
  int8_t lab8 = PTM_ALLOY_NONE;
  if (d.species && (S == 1 || S == 4)) {
    const int8_t c = __ldg(d.species + a);
    auto same = [&](int sl) { return __ldg(d.species + sm.NID(nib(cp, 15 - sl) - 1)) == c; };
    if (S == 1) {          // FCC: slots 1-4 in z = 0, 5-8 in y = 0, 9-12 in x = 0
      int sp = 0, op = 0;
      for (int p = 0; p < 3; p++) {
        int n = 0;
        for (int sl = 1 + 4 * p; sl <= 4 + 4 * p; sl++) n += same(sl);
        sp += n == 4;
        op += n == 0;
      }
      if (sp == 3) lab8 = PTM_ALLOY_PURE;
      else if (sp == 1 && op == 2) lab8 = PTM_ALLOY_L10;
      else if (sp == 2 && op == 1) lab8 = PTM_ALLOY_L12_MAJ;
      else if (op == 3) lab8 = PTM_ALLOY_L12_MIN;
    } else {               // BCC: slots 1-8 first shell, 9-14 second shell
      int in = 0, out = 0;
      for (int sl = 1; sl <= 8; sl++) in += same(sl);
      for (int sl = 9; sl <= 14; sl++) out += same(sl);
      if (in == 8 && out == 6) lab8 = PTM_ALLOY_PURE;
      else if (in == 0 && out == 6) lab8 = PTM_ALLOY_B2;
    }
  }
  return lab8;
}

__device__ void finalize(const FrameDesc &d, const Scratch &sm, const float4 *tplw, const Best &bst, int idi) {
  const int K = bst.K;
  const uint64_t lab = bst.lam(K);
  const uint64_t cand = __ldg((const unsigned long long *)&ptm_cand[bst.cand]);
  const int S = (int)(cand >> 60) & 7;
  float Sm[3][3];
  cov_matrix(K, sm, tplw, S, lab, cand, Sm);
  float mx, my, mz, Gv;
  data_moments(K, sm, mx, my, mz, Gv);
  const float Gw = __ldg(tplw + S * 15).w;
  float lam, q[4];
  {
    Qcp<float> o;
    qcp_solve<float>(Sm, Gv, Gw, o);
    float B = sqrtf(Gv * Gw);
    if (bst.fp64 || !(o.dP / (B * B * B) >= PTM_GAP)) {
      double S64[3][3];
      for (int a = 0; a < 3; a++) for (int b = 0; b < 3; b++) S64[a][b] = Sm[a][b];
      Qcp<double> o64;
      qcp_solve<double>(S64, (double)Gv, (double)Gw, o64);
      double q64[4];
      qcp_quat<double>(o64.K, o64.lam, q64);
      lam = (float)o64.lam;
      for (int i = 0; i < 4; i++) q[i] = (float)q64[i];
    } else {
      qcp_quat<float>(o.K, o.lam, q);
      lam = o.lam;
    }
  }
  const float s = lam / Gv;
  float R[3][3];
  quat_matrix<float>(q, R);
  // explicit residual of Eq. 3 at the optimum (avoids the cancellation of the
  // closed form near RMSD 0); the centre pairs with template slot 0 (origin)
  float r2 = 0.f;
  {
    float ux = -s * mx, uy = -s * my, uz = -s * mz;
    r2 = ux * ux + uy * uy + uz * uz;
  }
  float lsum = sqrtf(mx * mx + my * my + mz * mz);
  uint64_t corr = 0;
#pragma unroll 1
  for (int j = 0; j < K; j++) {
    int slot = nib(cand, nib(lab, j) - 1);
    float4 w = __ldg(tplw + S * 15 + slot);
    float vx = sm.DX(j) - mx, vy = sm.DY(j) - my, vz = sm.DZ(j) - mz;
    float rx = R[0][0] * w.x + R[0][1] * w.y + R[0][2] * w.z;
    float ry = R[1][0] * w.x + R[1][1] * w.y + R[1][2] * w.z;
    float rz = R[2][0] * w.x + R[2][1] * w.y + R[2][2] * w.z;
    float ex = s * vx - rx, ey = s * vy - ry, ez = s * vz - rz;
    r2 += ex * ex + ey * ey + ez * ez;
    lsum += sqrtf(vx * vx + vy * vy + vz * vz);
    corr |= (uint64_t)(j + 1) << (4 * (15 - slot));
  }
  const float rmsd = sqrtf(r2 / (float)(K + 1));
  const int64_t a = idi;
  if (!(rmsd <= d.rmsd_max)) {
    // unmatched after the RMSD_max cut (Sec. 5.1)
    if (d.structure) d.structure[a] = PTM_NONE;
    if (d.alloy) d.alloy[a] = PTM_ALLOY_NONE;
    if (d.rmsd) d.rmsd[a] = INFINITY;
    if (d.scale) d.scale[a] = 0.f;
    if (d.quat) { d.quat[4 * a] = 1.f; d.quat[4 * a + 1] = 0.f; d.quat[4 * a + 2] = 0.f; d.quat[4 * a + 3] = 0.f; }
    if (d.strain) for (int i = 0; i < 9; i++) d.strain[9 * a + i] = 0.f;
    if (d.corr) for (int i = 0; i < 15; i++) d.corr[15 * a + i] = -1;
    if (d.vm) d.vm[a] = 0.f;
    if (d.rf) for (int i = 0; i < 3; i++) d.rf[3 * a + i] = 0.f;
    return;
  }
  count(d, C_MATCHED);
  // correspondence: smallest member of its orbit (R12), atom ids per slot
  const uint64_t cp = canonical_corr(S, K, corr);
  if (d.structure) d.structure[a] = (int8_t)(S + 1);
  if (d.rmsd) d.rmsd[a] = rmsd;
  if (d.scale) d.scale[a] = s;
  if (d.corr) {
    d.corr[15 * a] = idi;
    for (int sl = 1; sl < 15; sl++) d.corr[15 * a + sl] = sl <= K ? sm.NID(nib(cp, 15 - sl) - 1) : -1;
  }
  // orientation in the fundamental zone: the equivalent rotation Q g with the
  // largest |w| (smallest angle); ties keep the earlier group element (Sec. 7)
  if (d.quat || d.rf) {
    float bw = -1.f, bq[4] = {1.f, 0.f, 0.f, 0.f};
    for (int g = ptm_group_off[S]; g < ptm_group_off[S + 1]; g++) {
      const float *gq = ptm_group_quat[g];
      float o0 = q[0] * gq[0] - q[1] * gq[1] - q[2] * gq[2] - q[3] * gq[3];
      if (fabsf(o0) > bw) {
        bw = fabsf(o0);
        bq[0] = o0;
        bq[1] = q[0] * gq[1] + q[1] * gq[0] + q[2] * gq[3] - q[3] * gq[2];
        bq[2] = q[0] * gq[2] - q[1] * gq[3] + q[2] * gq[0] + q[3] * gq[1];
        bq[3] = q[0] * gq[3] + q[1] * gq[2] - q[2] * gq[1] + q[3] * gq[0];
      }
    }
    float sg = bq[0] < 0.f ? -1.f : 1.f;
    if (d.quat) for (int i = 0; i < 4; i++) d.quat[4 * a + i] = sg * bq[i];
    // Rodrigues-Frank vector of the fundamental-zone orientation (Sec. 7)
    if (d.rf) for (int i = 0; i < 3; i++) d.rf[3 * a + i] = (sg * bq[i + 1]) / (sg * bq[0]);
  }
  // strain (Sec. 8, Eq. 6-7): both sets barycentred and scaled to mean distance
  // 1; the isotropic templates give pinv(V) = V^T / (G_w / 3), so
  // A = 3 S^T / (G_w l_data); then P = (A A^T)^(1/2), U proper.
  if (d.strain || d.vm) {
    const float ldat = lsum / (float)(K + 1);
    const float f = 3.f / (Gw * ldat);
    float A[3][3], AA[3][3], X[3][3];
    for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) A[i][j] = f * Sm[j][i];
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) AA[i][j] = A[i][0] * A[j][0] + A[i][1] * A[j][1] + A[i][2] * A[j][2];
    jacobi3(AA, X);
    float s0 = sqrtf(fmaxf(AA[0][0], 0.f)), s1 = sqrtf(fmaxf(AA[1][1], 0.f)), s2 = sqrtf(fmaxf(AA[2][2], 0.f));
    if (det3<float>(A) < 0.f) {         // U must stay proper: flip the smallest singular value
      if (s0 <= s1 && s0 <= s2) s0 = -s0;
      else if (s1 <= s2) s1 = -s1;
      else s2 = -s2;
    }
    const float sig[3] = {s0, s1, s2};
    float P[3][3];
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++)
        P[i][j] = X[i][0] * sig[0] * X[j][0] + X[i][1] * sig[1] * X[j][1] + X[i][2] * sig[2] * X[j][2];
    if (d.strain) for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) d.strain[9 * a + 3 * i + j] = P[i][j];
    // von Mises shear strain (Sec. 8) in its deviatoric form, equal to
    // 3/2 sum P_ij^2 - 1/2 (tr P)^2 but free of its cancellation near P = I
    if (d.vm) {
      const float t = (P[0][0] + P[1][1] + P[2][2]) / 3.f;
      const float e0 = P[0][0] - t, e1 = P[1][1] - t, e2 = P[2][2] - t;
      const float off = P[0][1] * P[0][1] + P[0][2] * P[0][2] + P[1][2] * P[1][2] +
                        P[1][0] * P[1][0] + P[2][0] * P[2][0] + P[2][1] * P[2][1];
      d.vm[a] = sqrtf(1.5f * (e0 * e0 + e1 * e1 + e2 * e2 + off));
    }
  }
  if (d.alloy) d.alloy[a] = alloy_label(d, sm, S, cp, a);
}

__device__ void write_unmatched(const FrameDesc &d, int64_t a) {
  if (d.structure) d.structure[a] = PTM_NONE;
  if (d.alloy) d.alloy[a] = PTM_ALLOY_NONE;
  if (d.rmsd) d.rmsd[a] = INFINITY;
  if (d.scale) d.scale[a] = 0.f;
  if (d.quat) { d.quat[4 * a] = 1.f; d.quat[4 * a + 1] = 0.f; d.quat[4 * a + 2] = 0.f; d.quat[4 * a + 3] = 0.f; }
  if (d.strain) for (int i = 0; i < 9; i++) d.strain[9 * a + i] = 0.f;
  if (d.corr) for (int i = 0; i < 15; i++) d.corr[15 * a + i] = -1;
  if (d.vm) d.vm[a] = 0.f;
  if (d.rf) for (int i = 0; i < 3; i++) d.rf[3 * a + i] = 0.f;
}

// Outputs of the winner in the FP64 form: the same steps as finalize, every
// metric quantity in FP64 from the FP64 neighbour vectors (results rounded to
// FP32 only when stored).
__device__ __noinline__ void finalize_fp64(const FrameDesc &d, const Scratch &sm, int K, uint64_t lab, int ci,
                                           const double (&ex)[PTM_KNN], const double (&ey)[PTM_KNN],
                                           const double (&ez)[PTM_KNN], int idi) {
  const uint64_t cand = ptm_cand[ci];
  const int S = (int)(cand >> 60) & 7;
  double m[3] = {0, 0, 0}, g = 0;
  for (int j = 0; j < K; j++) { m[0] += ex[j]; m[1] += ey[j]; m[2] += ez[j]; g += ex[j] * ex[j] + ey[j] * ey[j] + ez[j] * ez[j]; }
  for (int c = 0; c < 3; c++) m[c] /= (K + 1);
  const double Gv = g - (K + 1) * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  double Sm[3][3] = {{0}}, Gw = 0;
  for (int j = 0; j < K; j++) {
    const double *w = ptm_tpl64[S][nib(cand, nib(lab, j) - 1)];
    Sm[0][0] += w[0] * ex[j]; Sm[0][1] += w[0] * ey[j]; Sm[0][2] += w[0] * ez[j];
    Sm[1][0] += w[1] * ex[j]; Sm[1][1] += w[1] * ey[j]; Sm[1][2] += w[1] * ez[j];
    Sm[2][0] += w[2] * ex[j]; Sm[2][1] += w[2] * ey[j]; Sm[2][2] += w[2] * ez[j];
  }
  for (int slot = 0; slot <= K; slot++)
    Gw += ptm_tpl64[S][slot][0] * ptm_tpl64[S][slot][0] + ptm_tpl64[S][slot][1] * ptm_tpl64[S][slot][1] +
          ptm_tpl64[S][slot][2] * ptm_tpl64[S][slot][2];
  Qcp<double> o;
  qcp_solve<double>(Sm, Gv, Gw, o);
  double q[4], R[3][3];
  qcp_quat<double>(o.K, o.lam, q);
  const double s = o.lam / Gv;
  quat_matrix<double>(q, R);
  // explicit residual of Eq. 3; the centre pairs with template slot 0 (origin)
  double r2 = s * s * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  double lsum = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  uint64_t corr = 0;
  for (int j = 0; j < K; j++) {
    const int slot = nib(cand, nib(lab, j) - 1);
    const double *w = ptm_tpl64[S][slot];
    const double vx = ex[j] - m[0], vy = ey[j] - m[1], vz = ez[j] - m[2];
    const double rx = R[0][0] * w[0] + R[0][1] * w[1] + R[0][2] * w[2];
    const double ry = R[1][0] * w[0] + R[1][1] * w[1] + R[1][2] * w[2];
    const double rz = R[2][0] * w[0] + R[2][1] * w[1] + R[2][2] * w[2];
    const double dx = s * vx - rx, dy = s * vy - ry, dz = s * vz - rz;
    r2 += dx * dx + dy * dy + dz * dz;
    lsum += sqrt(vx * vx + vy * vy + vz * vz);
    corr |= (uint64_t)(j + 1) << (4 * (15 - slot));
  }
  const double rmsd = sqrt(r2 / (K + 1));
  const int64_t a = idi;
  if (!(rmsd <= d.rmsd_max)) { write_unmatched(d, a); return; }
  count(d, C_MATCHED);
  const uint64_t cp = canonical_corr(S, K, corr);
  if (d.structure) d.structure[a] = (int8_t)(S + 1);
  if (d.rmsd) d.rmsd[a] = (float)rmsd;
  if (d.scale) d.scale[a] = (float)s;
  if (d.corr) {
    d.corr[15 * a] = idi;
    for (int sl = 1; sl < 15; sl++) d.corr[15 * a + sl] = sl <= K ? sm.NID(nib(cp, 15 - sl) - 1) : -1;
  }
  if (d.quat || d.rf) {
    double bw = -1.0, bq[4] = {1.0, 0.0, 0.0, 0.0};
    for (int gi = ptm_group_off[S]; gi < ptm_group_off[S + 1]; gi++) {
      const float *gq = ptm_group_quat[gi];
      const double o0 = q[0] * gq[0] - q[1] * gq[1] - q[2] * gq[2] - q[3] * gq[3];
      if (fabs(o0) > bw) {
        bw = fabs(o0);
        bq[0] = o0;
        bq[1] = q[0] * gq[1] + q[1] * gq[0] + q[2] * gq[3] - q[3] * gq[2];
        bq[2] = q[0] * gq[2] - q[1] * gq[3] + q[2] * gq[0] + q[3] * gq[1];
        bq[3] = q[0] * gq[3] + q[1] * gq[2] - q[2] * gq[1] + q[3] * gq[0];
      }
    }
    const double sg = bq[0] < 0.0 ? -1.0 : 1.0;
    if (d.quat) for (int i = 0; i < 4; i++) d.quat[4 * a + i] = (float)(sg * bq[i]);
    if (d.rf) for (int i = 0; i < 3; i++) d.rf[3 * a + i] = (float)((sg * bq[i + 1]) / (sg * bq[0]));
  }
  if (d.strain || d.vm) {
    const double f = 3.0 / (Gw * (lsum / (K + 1)));
    double A[3][3], AA[3][3], X[3][3];
    for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) A[i][j] = f * Sm[j][i];
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) AA[i][j] = A[i][0] * A[j][0] + A[i][1] * A[j][1] + A[i][2] * A[j][2];
    jacobi3(AA, X);
    double sg[3] = {sqrt(fmax(AA[0][0], 0.0)), sqrt(fmax(AA[1][1], 0.0)), sqrt(fmax(AA[2][2], 0.0))};
    if (det3<double>(A) < 0.0) {
      const int k = (sg[0] <= sg[1] && sg[0] <= sg[2]) ? 0 : (sg[1] <= sg[2] ? 1 : 2);
      sg[k] = -sg[k];
    }
    double P[3][3];
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) P[i][j] = X[i][0] * sg[0] * X[j][0] + X[i][1] * sg[1] * X[j][1] + X[i][2] * sg[2] * X[j][2];
    if (d.strain) for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) d.strain[9 * a + 3 * i + j] = (float)P[i][j];
    if (d.vm) {
      const double t = (P[0][0] + P[1][1] + P[2][2]) / 3.0;
      const double e0 = P[0][0] - t, e1 = P[1][1] - t, e2 = P[2][2] - t;
      const double off = P[0][1] * P[0][1] + P[0][2] * P[0][2] + P[1][2] * P[1][2] +
                         P[1][0] * P[1][0] + P[2][0] * P[2][0] + P[2][1] * P[2][1];
      d.vm[a] = (float)sqrt(1.5 * (e0 * e0 + e1 * e1 + e2 * e2 + off));
    }
  }
  if (d.alloy) d.alloy[a] = alloy_label(d, sm, S, cp, a);
}

// Neighbour vectors for the metric steps, in rows DX / DY / DZ over the
// quantised copy (the hulls are done with it), and the neighbours' atom ids in
// row NID over their sorted indices: the contract values, or for a shifted
// image an error-free FP32 sum of difference and shift.
template <bool F64>
__device__ __forceinline__ void metric_vectors(const FrameDesc &d, const Scratch &sm, const int2 *nb, int64_t nst,
                                               typename RT<F64>::T xi, typename RT<F64>::T yi,
                                               typename RT<F64>::T zi) {
  typedef typename RT<F64>::T T;
#pragma unroll 7
  for (int t = 0; t < PTM_KNN; t++) {
    const int2 e = __ldg(nb + t * nst);
    if (e.x < 0) { sm.NID(t) = -1; sm.DX(t) = sm.DY(t) = sm.DZ(t) = 0.f; continue; }
    T xj, yj, zj;
    int idj;
    load_atom<F64>(d, e.x, xj, yj, zj, idj);
    sm.NID(t) = idj;
    int a0, a1, a2;
    img_unpack(e.y, a0, a1, a2);
    if constexpr (F64) {
      T sx, sy, sz;
      contract_shift<F64>(d, a0, a1, a2, sx, sy, sz);
      sm.DX(t) = (float)contract_dr(xj, xi, sx); sm.DY(t) = (float)contract_dr(yj, yi, sy);
      sm.DZ(t) = (float)contract_dr(zj, zi, sz);
    } else if (a0 == 0 && a1 == 0 && a2 == 0) {
      sm.DX(t) = __fsub_rn(xj, xi); sm.DY(t) = __fsub_rn(yj, yi); sm.DZ(t) = __fsub_rn(zj, zi);
    } else {
      float hx, hy, hz, lx, ly, lz;
      shift_f32(d, a0, a1, a2, hx, hy, hz, lx, ly, lz);
      float p, e1, q2, e2;
      two_sum(xj, -xi, p, e1); two_sum(p, hx, q2, e2); sm.DX(t) = q2 + (e1 + (e2 + lx));
      two_sum(yj, -yi, p, e1); two_sum(p, hy, q2, e2); sm.DY(t) = q2 + (e1 + (e2 + ly));
      two_sum(zj, -zi, p, e1); two_sum(p, hz, q2, e2); sm.DZ(t) = q2 + (e1 + (e2 + lz));
    }
  }
}

// FP64 contract vector of neighbour (sorted slot js, packed image img) of an
// atom at (xi, yi, zi), float32 positions.
__device__ __forceinline__ void vec64_row(const FrameDesc &d, float xi, float yi, float zi, int js, int img,
                                          double (&v)[3]) {
  float xj, yj, zj;
  int idj;
  load_atom<false>(d, js, xj, yj, zj, idj);
  int a0, a1, a2;
  img_unpack(img, a0, a1, a2);
  double hx, hy, hz;
  shift_f64(d, a0, a1, a2, hx, hy, hz);
  v[0] = contract_dr((double)xj, (double)xi, hx);
  v[1] = contract_dr((double)yj, (double)yi, hy);
  v[2] = contract_dr((double)zj, (double)zi, hz);
}

// Quantisation of the neighbours in `wide` (float32 input, rare): the frexp
// exponent of their largest FP64 vector component (-100000 if all are zero),
// then q = rint(dr 2^shift) into the Q rows.  Neighbour t of the atom is the
// list entry nb[t * nst]; the Q rows are per-thread columns of shared memory
// with stride PTM_BLOCK.
__device__ __noinline__ int wide_exponent(const FrameDesc &d, float xi, float yi, float zi, const int2 *nb,
                                          int64_t nst, uint32_t wide) {
  int e64 = -100000;
  for (; wide; wide &= wide - 1) {
    const int t = __ffs(wide) - 1;
    const int2 e = __ldg(nb + t * nst);
    double v[3];
    vec64_row(d, xi, yi, zi, e.x, e.y, v);
    const double m = fmax(fabs(v[0]), fmax(fabs(v[1]), fabs(v[2])));
    if (m > 0.0) { int et; frexp(m, &et); e64 = max(e64, et); }
  }
  return e64;
}

__device__ __noinline__ void wide_quantise(const FrameDesc &d, float xi, float yi, float zi, const int2 *nb,
                                           int64_t nst, float *q, uint32_t wide, int shift) {
  const double sc = ldexp(1.0, shift);
  for (; wide; wide &= wide - 1) {
    const int t = __ffs(wide) - 1;
    const int2 e = __ldg(nb + t * nst);
    double v[3];
    vec64_row(d, xi, yi, zi, e.x, e.y, v);
    for (int c = 0; c < 3; c++) q[(3 * t + c) * PTM_BLOCK] = (float)__double2int_rn(v[c] * sc);
  }
}

// ------------------------------------------------------------ one atom
// The method for one atom runs in two kernels.  k_hulls: neighbour vectors
// from the list, their quantised copy, the incremental hull and at k = 6, 12,
// 14 the Weinberg code and template lookup; it leaves, per atom, the matched
// snapshots' labellings and table entries (d.lam, d.ents).  k_match: QCP of
// every admissible correspondence, selection and the outputs.  `live` holds
// the lanes of this warp that entered together (all reach the warp-synchronous
// points below).

// Table entries of the snapshots k = 6, 12, 14, each + 1 in 10 bits (0 = none).
__device__ __forceinline__ uint32_t pack_ents(int e6, int e12, int e14) {
  return (uint32_t)(e6 + 1) | (uint32_t)(e12 + 1) << 10 | (uint32_t)(e14 + 1) << 20;
}

template <bool F64>
__device__ void hull_atom(const FrameDesc &d, int s, const Scratch &sm, unsigned live) {
  typedef typename RT<F64>::T T;
  T xi, yi, zi;
  int idi;
  load_atom<F64>(d, s, xi, yi, zi, idi);
  count(d, C_ATOMS);
  const int64_t sl = s - d.atom_offset;          // frame-local slot

  // ---- neighbours (Sec. 3): the list written by k_knn or k_topo, read in
  // place (entry t at nb[t * n]; the valid entries form a prefix).
  // Quantised copy for the exact hull predicates: q = rint(dr 2^(19 - e))
  // (half to even) on the FP64 contract vectors dr, 2^(e-1) <= max |dr_c| < 2^e
  const int2 *nb = d.nbr + sl;
  const int64_t nst = d.n;
  int cnt = 0;
  unsigned hmask;
  {
    if constexpr (F64) {
      T emax = 0;
#pragma unroll 1
      for (int t = 0; t < PTM_KNN; t++) {
        const int2 e = __ldg(nb + t * nst);
        if (e.x < 0) continue;
        cnt++;
        T xj, yj, zj;
        int idj;
        load_atom<F64>(d, e.x, xj, yj, zj, idj);
        int a0, a1, a2;
        img_unpack(e.y, a0, a1, a2);
        T sx, sy, sz;
        contract_shift<F64>(d, a0, a1, a2, sx, sy, sz);
        T cx = contract_dr(xj, xi, sx), cy = contract_dr(yj, yi, sy), cz = contract_dr(zj, zi, sz);
        emax = fmax(emax, fmax(fabs(cx), fmax(fabs(cy), fabs(cz))));
      }
      int e;
      frexp(emax, &e);
      const T sc = (T)ldexp(1.0, PTM_QBITS - e);
#pragma unroll 1
      for (int t = 0; t < PTM_KNN; t++) {
        if (t >= cnt) continue;
        const int2 en = __ldg(nb + t * nst);
        T xj, yj, zj;
        int idj;
        load_atom<F64>(d, en.x, xj, yj, zj, idj);
        int a0, a1, a2;
        img_unpack(en.y, a0, a1, a2);
        T sx, sy, sz;
        contract_shift<F64>(d, a0, a1, a2, sx, sy, sz);
        T cx = contract_dr(xj, xi, sx), cy = contract_dr(yj, yi, sy), cz = contract_dr(zj, zi, sz);
        sm.Q(t, 0) = (float)__double2int_rn(cx * sc); sm.Q(t, 1) = (float)__double2int_rn(cy * sc);
        sm.Q(t, 2) = (float)__double2int_rn(cz * sc);
      }
    } else {
      // float32 input: a neighbour in the same image whose FP32 differences
      // are exact (Sterbenz: |x_j - x_i| below min(|x_i|, |x_j|)) has its FP64
      // vector in FP32 already, kept in the Q rows between the two loops; the
      // others (bit t of `wide`: shifted images, atoms near a coordinate plane
      // through the origin) are evaluated in FP64 out of line
      float emaxf = 0.f;
      uint32_t wide = 0;
#pragma unroll 7
      for (int t = 0; t < PTM_KNN; t++) {
        const int2 e = __ldg(nb + t * nst);
        if (e.x < 0) continue;
        cnt++;
        float xj, yj, zj;
        int idj;
        load_atom<false>(d, e.x, xj, yj, zj, idj);
        const float px = __fsub_rn(xj, xi), py = __fsub_rn(yj, yi), pz = __fsub_rn(zj, zi);
        const bool exact = e.y == img_pack(0, 0, 0) && fabsf(px) < fminf(fabsf(xi), fabsf(xj)) &&
                           fabsf(py) < fminf(fabsf(yi), fabsf(yj)) && fabsf(pz) < fminf(fabsf(zi), fabsf(zj));
        sm.Q(t, 0) = px; sm.Q(t, 1) = py; sm.Q(t, 2) = pz;
        if (exact) emaxf = fmaxf(emaxf, fmaxf(fabsf(px), fmaxf(fabsf(py), fabsf(pz))));
        else wide |= 1u << t;
      }
      int e;
      frexpf(emaxf, &e);
      if (wide) {
        const int e64 = wide_exponent(d, xi, yi, zi, nb, nst, wide);
        if (e64 > -100000) e = emaxf > 0.f ? max(e, e64) : e64;
      }
      const float sc = ldexpf(1.f, PTM_QBITS - e);
#pragma unroll
      for (int t = 0; t < PTM_KNN; t++) {
        if (t >= cnt || (wide >> t & 1)) continue;
        sm.Q(t, 0) = rintf(sm.Q(t, 0) * sc); sm.Q(t, 1) = rintf(sm.Q(t, 1) * sc); sm.Q(t, 2) = rintf(sm.Q(t, 2) * sc);
      }
      if (wide) wide_quantise(d, xi, yi, zi, nb, nst, sm.q + sm.t, wide, PTM_QBITS - e);
    }
    hmask = __ballot_sync(live, cnt >= 4);       // lanes that go on to the hulls
    if (cnt < 4) { d.ents[sl] = 0; return; }
  }

  // ---- hulls of the first 6, 12, 14 neighbours, built incrementally (Sec. 4)
  Best bst;
  bst.ent6 = bst.ent12 = bst.ent14 = -1;
  bst.lam6 = bst.lam12 = bst.lam14 = 0;
  const uint32_t mask = d.mask;
  int kmax = (mask & 16) ? 14 : ((mask & 14) ? 12 : 6);
  kmax = min(kmax, cnt);
  bool alive = kmax >= 6;
  int nf = alive ? hull_init(sm, d) : 0;
  for (int p = 4; p <= PTM_KNN; p++) {
    // every insertion step starts warp-converged: a lane that finished (or took
    // a snapshot's longer path) waits here instead of drifting into a later
    // step alone, so the visibility tests, walks and QCP loops keep full warps
    if (!__any_sync(hmask, alive)) break;
    // the hull now holds neighbours 0..p-1: complete for K = 6, 12, 14.  The
    // centre test of a snapshot rides on the visibility test of point p.
    const bool want = (p == 6 && (mask & 1)) || (p == 12 && (mask & 14)) || (p == 14 && (mask & 16));
    bool centre_in = false;
    uint32_t vis = 0;
    const unsigned vmask = __ballot_sync(hmask, alive && p < kmax);          // lanes testing point p
    const unsigned cmask = __ballot_sync(hmask, alive && p >= kmax && want); // lanes testing only the centre
    if (alive) {
      if (p < kmax) vis = hull_visibility(sm, nf, p, want, centre_in, vmask, d);
      else if (want) centre_in = hull_centre_inside(sm, nf, cmask, d);
    }
    if (alive && want && centre_in) snapshot(p, sm, d, nf, bst);
    if (!alive) continue;
    if (p == kmax || !vis) { alive = false; continue; }   // done, or p lies inside the hull
    nf = hull_apply(sm, nf, vis, p, d);
    if (nf < 0) alive = false;
  }
  d.ents[sl] = pack_ents(bst.ent6, bst.ent12, bst.ent14);
  if (bst.ent6 >= 0) d.lam[sl] = bst.lam6;
  if (bst.ent12 >= 0) d.lam[d.n + sl] = bst.lam12;
  if (bst.ent14 >= 0) d.lam[2 * d.n + sl] = bst.lam14;
}

// P64 selects the FP64 form: every candidate scored and the winner's outputs
// computed in FP64 (the one-frame-per-launch comparison form).
template <bool F64, bool P64 = false>
__device__ void match_atom(const FrameDesc &d, int s, const Scratch &sm, const float4 *tplw, unsigned live) {
  typedef typename RT<F64>::T T;
  const int64_t sl = s - d.atom_offset;
  const uint32_t ents = __ldg(d.ents + sl);
  const unsigned qmask = __ballot_sync(live, ents != 0);
  T xi, yi, zi;
  int idi;
  load_atom<F64>(d, s, xi, yi, zi, idi);
  if (!ents) { write_unmatched(d, idi); return; }
  Best bst;
  bst.b1 = bst.b2 = INFINITY;
  bst.K = -1; bst.cand = -1; bst.fp64 = 0;
  bst.ent6 = (int)(ents & 1023) - 1;
  bst.ent12 = (int)(ents >> 10 & 1023) - 1;
  bst.ent14 = (int)(ents >> 20 & 1023) - 1;
  bst.lam6 = bst.ent6 >= 0 ? __ldg((const unsigned long long *)d.lam + sl) : 0;
  bst.lam12 = bst.ent12 >= 0 ? __ldg((const unsigned long long *)d.lam + d.n + sl) : 0;
  bst.lam14 = bst.ent14 >= 0 ? __ldg((const unsigned long long *)d.lam + 2 * d.n + sl) : 0;
  const int2 *nb = d.nbr + sl;                   // the neighbour list, entry t at nb[t * n]
  const int64_t nst = d.n;
  double ex[P64 ? PTM_KNN : 1], ey[P64 ? PTM_KNN : 1], ez[P64 ? PTM_KNN : 1];
  if constexpr (P64) {
    for (int t = 0; t < PTM_KNN; t++) {
      const int2 e = __ldg(nb + t * nst);
      if (e.x < 0) break;                          // the valid entries form a prefix
      vec_fp64<F64>(d, xi, yi, zi, e.x, e.y, ex[t], ey[t], ez[t]);
    }
  }
  metric_vectors<F64>(d, sm, nb, nst, xi, yi, zi);
  if constexpr (!P64) {
    score_candidates(d, sm, tplw, bst, qmask);
    if (bst.K < 0) { write_unmatched(d, idi); return; }     // every match masked out
  } else {
    int ns = 0;
    const int w = select_fp64(d, bst, ex, ey, ez, &ns);
    if (ns) { count(d, C_CAND, ns); }
    if (w < 0) { write_unmatched(d, idi); return; }
    const int K = w >> 16;
    finalize_fp64(d, sm, K, bst.lam(K), w & 0xffff, ex, ey, ez, idi);
    return;
  }
  if (bst.b2 <= bst.b1 + PTM_BAND) {
    count(d, C_TIE64);
    const int w = rerank_fp64<F64>(d, s, bst);
    if (w >= 0) { bst.K = w >> 16; bst.cand = w & 0xffff; }
  }
  finalize(d, sm, tplw, bst, idi);
}

// ------------------------------------------------------------------ kernels
// Copies a frame's shift tables, passed by value, into device memory: stream
// ordered, so back-to-back asynchronous calls never share a host staging buffer.
__global__ void k_put_tables(const __grid_constant__ ShiftTables t, ShiftTables *out) {
  const float *src = reinterpret_cast<const float *>(&t);
  float *dst = reinterpret_cast<float *>(out);
  for (int i = threadIdx.x; i < (int)(sizeof(ShiftTables) / 4); i += blockDim.x) dst[i] = src[i];
}

struct BinParams {
  float Hinv[9];     // fractional = x . Hinv
  float W[3];        // perpendicular cell widths
  int nb[3];
  int pbc[3];
  int64_t n;
  int f64;
  // batches only: where this frame lives
  const void *pos;   // the frame's positions
  int *dstat;        // the frame's status words
  unsigned long long *counters;   // the call's counters (excluded atoms)
  int64_t atom_off;  // first atom of the frame in the batch order
  int cell_off;      // first cell of the frame in the batch's cell array
};

#define PTM_WRAP_TOL 1e-4f

// Cell of one atom of frame p (shared by the single-frame and batched
// binning), its lattice wrap (packed image) and how far it lies outside the
// cell (Angstrom, plus a rounding slack).  An atom with a non-finite
// coordinate, or more than PTM_FAR_PERIODS periods from the cell, is excluded:
// it gets the marker wrap PTM_EXCLUDED (no valid image packs to it), cell 0 and
// no overshoot, so it is nobody's neighbour and is itself left unmatched.
__device__ __forceinline__ int bin_atom(const BinParams &p, const void *pos, int64_t li, int &wrap, float &over) {
  float x, y, z;
  if (p.f64) {
    const double *q = (const double *)pos + 3 * li;
    x = (float)q[0]; y = (float)q[1]; z = (float)q[2];
  } else {
    const float *q = (const float *)pos + 3 * li;
    x = q[0]; y = q[1]; z = q[2];
  }
  int bc[3], w[3];
  over = 0.f;
  bool ok = true;
  for (int c = 0; c < 3; c++) {
    float f = x * p.Hinv[c] + y * p.Hinv[3 + c] + z * p.Hinv[6 + c];
    ok &= fabsf(f) < PTM_FAR_PERIODS;              // false for NaN and infinities too
    w[c] = 0;
    if (p.pbc[c] && (f < -PTM_WRAP_TOL || f >= 1.f + PTM_WRAP_TOL)) {
      w[c] = (int)floorf(f);
      f -= (float)w[c];
    }
    over = fmaxf(over, fmaxf(-f, f - 1.f) * p.W[c]);
    int b = (int)floorf(f * (float)p.nb[c]);
    bc[c] = min(max(b, 0), p.nb[c] - 1);
  }
  if (!ok) {
    wrap = PTM_EXCLUDED;
    over = 0.f;
    return 0;
  }
  // rounding of the fractional coordinates is covered by a small extra slack
  over = fmaxf(over, 0.f) + 1e-5f * fmaxf(p.W[0], fmaxf(p.W[1], p.W[2]));
  wrap = img_pack(w[0], w[1], w[2]);
  return (bc[0] * p.nb[1] + bc[1]) * p.nb[2] + bc[2];
}

__global__ void k_bin(const void *pos, BinParams p, int *cell_count, int *atom_cell, int *atom_rank,
                      int *atom_wrap, int *dstat) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  int wrap;
  float over;
  const int cell = bin_atom(p, pos, i, wrap, over);
  if (wrap == PTM_EXCLUDED) atomicAdd(p.counters + C_EXCLUDED, 1ull);
  else if (wrap != img_pack(0, 0, 0)) dstat[0] = 1;
  atomicMax(dstat + 1, __float_as_int(over));      // uniform address: the compiler aggregates per warp
  atom_cell[i] = cell;
  atom_rank[i] = atomicAdd(cell_count + cell, 1);
  atom_wrap[i] = wrap;
}

#define SCAN_BLOCK 1024
// exclusive scan, level 1: per-block scan of 2 elements per thread
__global__ void k_scan_block(const int *in, int *out, int *block_sums, int n) {
  __shared__ int sh[SCAN_BLOCK * 2];
  int base = blockIdx.x * SCAN_BLOCK * 2;
  int t = threadIdx.x;
  int a = base + 2 * t, b = a + 1;
  int va = a < n ? in[a] : 0, vb = b < n ? in[b] : 0;
  sh[2 * t] = va;
  sh[2 * t + 1] = va + vb;
  __syncthreads();
  // Hillis-Steele over the pair sums
  int v = sh[2 * t + 1];
  for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
    int add = t >= off ? sh[2 * (t - off) + 1] : 0;
    __syncthreads();
    v += add;
    sh[2 * t + 1] = v;
    __syncthreads();
  }
  int excl = v - (va + vb);
  if (a < n) out[a] = excl;
  if (b < n) out[b] = excl + va;
  if (t == SCAN_BLOCK - 1) block_sums[blockIdx.x] = v;
}

// level 2: one block scans the block sums serially in chunks
__global__ void k_scan_sums(int *block_sums, int nblocks, int *total_out) {
  __shared__ int sh[SCAN_BLOCK];
  int carry = 0;
  for (int base = 0; base < nblocks; base += SCAN_BLOCK) {
    int t = threadIdx.x, i = base + t;
    int v = i < nblocks ? block_sums[i] : 0;
    sh[t] = v;
    __syncthreads();
    for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
      int add = t >= off ? sh[t - off] : 0;
      __syncthreads();
      sh[t] += add;
      __syncthreads();
    }
    if (i < nblocks) block_sums[i] = carry + sh[t] - v;
    int tot = sh[SCAN_BLOCK - 1];
    __syncthreads();
    carry += tot;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(int *out, const int *block_sums, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += block_sums[i / (SCAN_BLOCK * 2)];
}

__global__ void k_scatter(const void *pos, int f64, int64_t n, const int *atom_cell, const int *atom_rank,
                          const int *atom_wrap, const int *cell_start, void *sorted, int *sbin, int *wrapv) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = atom_cell[i];
  int slot = cell_start[c] + atom_rank[i];
  if (f64) {
    const double *q = (const double *)pos + 3 * i;
    Atom64 a;
    a.x = q[0]; a.y = q[1]; a.z = q[2]; a.id = i;
    ((Atom64 *)sorted)[slot] = a;
  } else {
    const float *q = (const float *)pos + 3 * i;
    ((float4 *)sorted)[slot] = make_float4(q[0], q[1], q[2], __int_as_float((int)i));
  }
  sbin[slot] = c;
  wrapv[slot] = atom_wrap[i];
}

// ------------------------------------------------------------ batched frames
// Frame of batch atom i: the last frame whose first atom is <= i.
__device__ __forceinline__ int frame_of(const int64_t *atom_off, int nframes, int64_t i) {
  int lo = 0, hi = nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg((const unsigned long long *)atom_off + mid) <= (unsigned long long)i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_bin_batch(const BinParams *__restrict__ bp, const int64_t *__restrict__ atom_off, int nframes,
                            int64_t ntotal, int *cell_count, int *atom_cell, int *atom_rank, int *atom_wrap) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntotal) return;
  const int f = frame_of(atom_off, nframes, i);
  const BinParams &p = bp[f];
  int wrap;
  float over;
  const int cell = p.cell_off + bin_atom(p, p.pos, i - p.atom_off, wrap, over);
  if (wrap == PTM_EXCLUDED) atomicAdd(p.counters + C_EXCLUDED, 1ull);
  else if (wrap != img_pack(0, 0, 0)) p.dstat[0] = 1;
  // one atomic per frame per warp (over > 0, so its bits order as integers):
  // per-atom atomics on a frame's single status word serialise at the L2
  const unsigned same = __match_any_sync(__activemask(), f);
  const int omax = __reduce_max_sync(same, __float_as_int(over));
  if ((threadIdx.x & 31) == __ffs(same) - 1) atomicMax(p.dstat + 1, omax);
  atom_cell[i] = cell;
  atom_rank[i] = atomicAdd(cell_count + cell, 1);
  atom_wrap[i] = wrap;
}

__global__ void k_scatter_batch(const BinParams *__restrict__ bp, const int64_t *__restrict__ atom_off, int nframes,
                                int64_t ntotal, const int *atom_cell, const int *atom_rank, const int *atom_wrap,
                                const int *cell_start, void *sorted, int *sbin, int *wrapv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntotal) return;
  const int f = frame_of(atom_off, nframes, i);
  const BinParams &p = bp[f];
  const int64_t li = i - p.atom_off;
  const int c = atom_cell[i];
  const int slot = cell_start[c] + atom_rank[i];
  if (p.f64) {
    const double *q = (const double *)p.pos + 3 * li;
    Atom64 a;
    a.x = q[0]; a.y = q[1]; a.z = q[2]; a.id = li;
    ((Atom64 *)sorted)[slot] = a;
  } else {
    const float *q = (const float *)p.pos + 3 * li;
    ((float4 *)sorted)[slot] = make_float4(q[0], q[1], q[2], __int_as_float((int)li));
  }
  sbin[slot] = c - p.cell_off;
  wrapv[slot] = atom_wrap[i];
}

constexpr size_t atom_smem_bytes() { return (size_t)PTM_BLOCK * SCRATCH_WORDS * 4; }
// k_match keeps only the neighbour vectors (42 words) and the neighbours' atom
// ids (14 words) per thread; the images are read from the neighbour list
constexpr int MATCH_WORDS = 42 + 14;
constexpr size_t match_smem_bytes() { return (size_t)PTM_BLOCK * MATCH_WORDS * 4; }

// Resident blocks per SM of k_hulls: 8 x (98 words x 64 threads + the 1 KB the
// driver reserves per block) fits 228 KB of shared memory, and 8 x 64 threads x
// 128 registers the register file.
#define PTM_ATOM_BLOCKS_PER_SM 8
// k_match: 11 x (56 words x 64 threads + two descriptor copies + 1 KB) fits, at up
// to 93 registers
#define PTM_MATCH_BLOCKS_PER_SM 11
// Frames of a batch with at least this many atoms get a k_match launch of their
// own (on a 2^20-atom frame the persistent k_match_batch took 0.47 ms more than
// such a launch's 1.47 ms); the own launches alternate between the batch's stream and
// PTM_MATCH_SIDE_STREAMS side streams, so that each launch's last wave overlaps
// the next launch (the batch of 256 frames: matching 60.6 -> 48.8 ms)
#define PTM_MATCH_OWN_LAUNCH 65536
#define PTM_MATCH_SIDE_STREAMS 2

// Scratch rows of k_hulls in a block's dynamic shared memory (row layout of
// Scratch without the nid / img rows).
__device__ __forceinline__ Scratch scratch_rows(unsigned char *smem) {
  Scratch sm;
  sm.th = (uint64_t *)smem;
  sm.q = (float *)(sm.th + 14 * PTM_BLOCK);
  sm.nid = nullptr;                 // k_hulls reads the neighbour list in place
  sm.img = nullptr;
  sm.code = (uint32_t *)(sm.q + 42 * PTM_BLOCK);
  sm.fac = (uint16_t *)(sm.code + PTM_CODE_WORDS * PTM_BLOCK);
  sm.used = sm.fac + 24 * PTM_BLOCK;
  sm.t = threadIdx.x;
  return sm;
}

// The rows k_match uses (the others stay null).
__device__ __forceinline__ Scratch match_rows(unsigned char *smem) {
  Scratch sm;
  sm.th = nullptr; sm.code = nullptr; sm.fac = nullptr; sm.used = nullptr;
  sm.q = (float *)smem;
  sm.nid = (int *)(sm.q + 42 * PTM_BLOCK);
  sm.img = nullptr;                 // images are read from the neighbour list
  sm.t = threadIdx.x;
  return sm;
}

// Normalised templates as float4 (x, y, z, .) in global memory, read through the
// read-only cache (shared memory is spent on per-thread scratch).
__device__ __forceinline__ const float4 *template_rows() { return reinterpret_cast<const float4 *>(&ptm_tpl[0][0][0]); }

// The frame descriptor travels by value in the kernel parameters, so back-to-back
// asynchronous calls never share a staging buffer.
template <bool F64>
__global__ void __launch_bounds__(PTM_BLOCK, PTM_ATOM_BLOCKS_PER_SM) k_hulls(const __grid_constant__ FrameDesc d) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Scratch sm = scratch_rows(smem);
  const int64_t s = (int64_t)blockIdx.x * PTM_BLOCK + threadIdx.x;
  const unsigned live = __ballot_sync(0xffffffffu, s < d.n);
  if (s >= d.n) return;
  hull_atom<F64>(d, (int)s, sm, live);
}

template <bool F64, bool P64 = false>
__global__ void __launch_bounds__(PTM_BLOCK, PTM_MATCH_BLOCKS_PER_SM) k_match(const __grid_constant__ FrameDesc d) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Scratch sm = match_rows(smem);
  const float4 *tplw = template_rows();
  const int64_t s = (int64_t)blockIdx.x * PTM_BLOCK + threadIdx.x;     // frame-local slot
  const unsigned live = __ballot_sync(0xffffffffu, s < d.n);
  if (s >= d.n) return;
  match_atom<F64, P64>(d, (int)(s + d.atom_offset), sm, tplw, live);
}

// Neighbour lists of one frame (Euclidean order), one thread per atom.
template <bool F64>
__global__ void __launch_bounds__(PTM_KNN_BLOCK, PTM_KNN_BLOCKS_PER_SM) k_knn(const __grid_constant__ FrameDesc d) {
  extern __shared__ __align__(16) int knn_smem[];
  const int64_t s = (int64_t)blockIdx.x * PTM_KNN_BLOCK + threadIdx.x;
  if (s >= d.n) return;
  knn_atom<F64>(d, (int)s, knn_smem);
}

// The same over a batch: each slot finds its frame; frames in the topological
// order are left to k_topo_batch.
template <bool F64>
__global__ void __launch_bounds__(PTM_KNN_BLOCK, PTM_KNN_BATCH_BLOCKS_PER_SM)
    k_knn_batch(const FrameDesc *__restrict__ descs, const int64_t *__restrict__ atom_off, int nframes,
                int64_t ntotal) {
  extern __shared__ __align__(16) int knn_smem[];
  const int64_t s = (int64_t)blockIdx.x * PTM_KNN_BLOCK + threadIdx.x;
  if (s >= ntotal) return;
  const FrameDesc &d = descs[frame_of(atom_off, nframes, s)];
  if (d.ordering != PTM_ORDER_EUCLIDEAN) return;
  knn_atom<F64>(d, (int)s, knn_smem);
}

// Persistent per-atom passes over a batch: every warp pulls tiles of
// tile_atoms (a multiple of 32) consecutive slots from a global queue until the
// batch is exhausted, so uneven frames balance across the GPU and no warp waits
// for the other warp of its block.  The slots are the batch's sorted slots, or
// with a map (map_frames, map_off, nmap) a virtual numbering of the listed
// frames' atoms only: virtual slot v of listed frame k = frame_of(map_off, ...)
// is sorted slot atom_offset + v - map_off[k] of frame map_frames[k].  With
// `head` (this warp's slot of shared memory) a tile whose slots all belong to
// one frame reads that frame's descriptor from a shared copy, made when the
// frame changes.  fn(desc, slot, live).
template <typename Fn>
__device__ __forceinline__ void persistent_tiles(const FrameDesc *__restrict__ descs,
                                                 const int64_t *__restrict__ atom_off, int nframes, int64_t ntotal,
                                                 const int *__restrict__ map_frames, int tile_atoms,
                                                 unsigned long long *queue, FrameDesc *head, Fn &&fn) {
  const int lane = threadIdx.x & 31;
  int cached = -1;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(queue, (unsigned long long)tile_atoms);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((long long)base >= ntotal) break;
    for (int k = 0; k < tile_atoms; k += 32) {
      long long s = (long long)base + k + lane;
      const unsigned live = __ballot_sync(0xffffffffu, s < ntotal);
      if (!live) break;                  // the rest of a tile past the end (warp-uniform)
      int f = -1;
      if (s < ntotal) {
        f = frame_of(atom_off, nframes, s);
        if (map_frames) {
          s += (long long)__ldg((const long long *)&descs[__ldg(map_frames + f)].atom_offset) -
               (long long)__ldg((const long long *)atom_off + f);
          f = __ldg(map_frames + f);
        }
      }
      const FrameDesc *dp = descs + f;
      if (head) {
        const int f0 = __shfl_sync(0xffffffffu, f, 0);          // lane 0 is live whenever any lane is
        if (__all_sync(0xffffffffu, f == f0 || !(live >> lane & 1))) {
          if (f0 != cached) {
            const int *src = reinterpret_cast<const int *>(descs + f0);
            int *dst = reinterpret_cast<int *>(head);
            for (int w = lane; w < (int)(sizeof(FrameDesc) / 4); w += 32) dst[w] = __ldg(src + w);
            __syncwarp();
            cached = f0;
          }
          dp = head;
        }
      }
      if (live >> lane & 1) fn(*dp, (int)s, live);
    }
  }
}

template <bool F64>
__global__ void __launch_bounds__(PTM_BLOCK, PTM_ATOM_BLOCKS_PER_SM)
    k_hulls_batch(const FrameDesc *__restrict__ descs, const int64_t *__restrict__ atom_off, int nframes,
                  int64_t ntotal, int tile_atoms, unsigned long long *queue) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Scratch sm = scratch_rows(smem);
  persistent_tiles(descs, atom_off, nframes, ntotal, nullptr, tile_atoms, queue, nullptr,
                   [&](const FrameDesc &d, int s, unsigned live) { hull_atom<F64>(d, s, sm, live); });
}

// k_match over the atoms of the batch's smaller frames (the larger ones get a
// k_match launch each, with their descriptor in the kernel parameters): map_off
// is the prefix sum of the listed frames' sizes, map_frames their indices.
template <bool F64>
__global__ void __launch_bounds__(PTM_BLOCK, PTM_MATCH_BLOCKS_PER_SM)
    k_match_batch(const FrameDesc *__restrict__ descs, const int64_t *__restrict__ map_off,
                  const int *__restrict__ map_frames, int nmap, int64_t nslots, int tile_atoms,
                  unsigned long long *queue) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Scratch sm = match_rows(smem);
  const float4 *tplw = template_rows();
  __shared__ FrameDesc heads[PTM_BLOCK / 32];
  persistent_tiles(descs, map_off, nmap, nslots, map_frames, tile_atoms, queue, &heads[threadIdx.x >> 5],
                   [&](const FrameDesc &d, int s, unsigned live) { match_atom<F64, false>(d, s, sm, tplw, live); });
}

}  // namespace ptm

