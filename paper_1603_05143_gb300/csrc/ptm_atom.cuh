// Per-atom Polyhedral Template Matching pipeline, one thread per atom.
//
// Larsen, Schmidt & Schiotz, "Robust Structural Identification via Polyhedral
// Template Matching".  Steps per atom (Algorithm 1, Euclidean ordering):
//   kNN (k = 14) under the distance contract  (Sec. 3)
//   neighbour vectors, quantised copy for the exact hull predicates
//   ONE incremental convex hull over neighbours 1..14; the hulls of the first
//   6 and 12 neighbours are its intermediate states (Sec. 4)
//   at k = 6, 12, 14: centre-inside test, canonical Weinberg code, template lookup
//   QCP superposition of each admissible correspondence (Eq. 3-4)
//   selection, then orientation (Sec. 7), strain (Sec. 8) and alloy (Sec. 6).
//
// Per-thread scratch lives in shared memory laid out [word][thread], so every
// thread of a warp hits its own bank whatever index it uses.
#pragma once
#include <stdint.h>
#include <math.h>

#include "ptm_tables_gen.h"

#define PTM_BLOCK 64
#define PTM_KNN 14
#define PTM_QBITS 19
#define PTM_RMAX 6              // widest cell-search radius (in cells) before giving up
#define PTM_BAND 1e-5f          // FP32 RMSD^2 band inside which candidates are re-ranked in FP64
#define PTM_TIE 1e-12           // FP64 RMSD^2 tie window (earlier template, then smaller correspondence)
#define PTM_GAP 0.02f           // minimum normalised P'(lambda_1) / B^3 for an FP32 QCP solution

namespace ptm {

struct Atom64 { double x, y, z; long long id; };

// Shift n.H of each lattice image n in [-2,2]^3, in device memory beside the
// frame's descriptor: the FP64 value, its FP32 rounding and the FP32 rounding of
// the remainder (compensated neighbour vectors).
struct ShiftTables {
  float s32[125][3];
  float slo[125][3];
  double s64[125][3];
};

// Device-resident description of one frame (filled by the host).
struct FrameDesc {
  const void *sorted;          // float4 (x, y, z, id bits) or Atom64, cell-sorted (ids are frame-local)
  const int *sbin;             // frame-local cell of each sorted slot
  const int *cell_start;       // this frame's ncell + 1 offsets into sorted (global sorted indices)
  const int *wrapv;            // packed lattice wrap per sorted slot
  const int8_t *species;       // by atom id, or NULL
  const void *positions;       // caller positions (by atom id)
  int64_t n;
  int nb[3];
  int pbc[3];
  int f64;
  uint32_t mask;
  float rmsd_max;
  float min_cell_width;        // smallest perpendicular cell width (Angstrom)
  float smax;                  // bound on the length of an image shift n.H with |n_r| <= 1 (periodic r)
  double H[9];                 // rows = cell vectors
  const struct ShiftTables *tab;   // shifts of the images n in [-2,2]^3 (device memory)
  // outputs (by atom id)
  int8_t *structure;
  int8_t *alloy;
  float *rmsd;
  float *scale;
  float *quat;
  float *strain;
  int32_t *corr;
  float *vm;                   // derived: von Mises shear strain
  float *rf;                   // derived: Rodrigues-Frank vector
  const int2 *nbr;             // neighbour list: [t][n] (sorted slot, image) of neighbour t of the
                               // atom at frame-local slot s - atom_offset (slot -1: none), written
                               // by k_knn (Euclidean order) or k_topo (topological order)
  int ordering;                // PTM_ORDER_EUCLIDEAN or PTM_ORDER_TOPOLOGICAL
  uint64_t *lam;               // k_hulls -> k_match: [3][n] Weinberg labelling of snapshot k = 6, 12, 14
  uint32_t *ents;              // [n] their table entries + 1, 10 bits each (0: no match)
  int *dstat;                  // [0] any atom wrapped, [1] overshoot (float bits, Angstrom)
  unsigned long long *counters;  // the C_* counters below
  int64_t atom_offset;         // first sorted slot of this frame (0 for a single frame)
};

enum { C_ATOMS = 0, C_MATCHED, C_KNN_WIDE, C_KNN_FAIL, C_SOS, C_QCP64, C_TIE64, C_INTERNAL, C_CAND, C_CANDPTS, C_TOPO64,
       C_KNN64, C_EXCLUDED, C_NCOUNTERS };

__device__ __forceinline__ void count(const FrameDesc &d, int which, unsigned long long v = 1) {
  atomicAdd(d.counters + which, v);
}

// ------------------------------------------------------------ shared scratch
// Rows are [word][thread] (every lane its own bank).  In k_hulls the 42 rows of
// q hold the quantised neighbour vectors while the hulls are built, beside the
// rotation system, code, facet and edge rows: 98 words per thread let 8 blocks
// of 64 threads share an SM's 228 KB.  k_match uses only q (the FP32 metric
// vectors), nid (the neighbours' sorted indices, then their atom ids) and img.
struct Scratch {
  float *q;          // [42][B]  quantised neighbour vectors (integers |q| <= 2^19, exact in FP32),
                     //          then the metric vectors DX / DY / DZ
  int *nid;          // [14][B]  neighbour sorted index, then atom id (k_match)
  int *img;          // [14][B]  neighbour image (img_pack) (k_match)
  uint16_t *fac;     // [24][B]  hull facets a | b << 4 | c << 8 (ccw from outside)
  uint64_t *th;      // [14][B]  third vertex of directed edge u->v, nibble v of row u (0xF none)
  uint16_t *used;    // [14][B]  directed-edge bit rows (hull horizon, Weinberg walk)
  uint32_t *code;    // [9][B]   best Weinberg code so far from its third label on (nibbles)
  int t;             // thread index in block
  __device__ __forceinline__ float &Q(int p, int c) const { return q[(3 * p + c) * PTM_BLOCK + t]; }
  __device__ __forceinline__ int QI(int p, int c) const { return (int)q[(3 * p + c) * PTM_BLOCK + t]; }
  __device__ __forceinline__ float &DX(int j) const { return Q(j, 0); }
  __device__ __forceinline__ float &DY(int j) const { return Q(j, 1); }
  __device__ __forceinline__ float &DZ(int j) const { return Q(j, 2); }
  __device__ __forceinline__ int &NID(int j) const { return nid[j * PTM_BLOCK + t]; }
  __device__ __forceinline__ int &IMG(int j) const { return img[j * PTM_BLOCK + t]; }
  __device__ __forceinline__ uint16_t &F(int f) const { return fac[f * PTM_BLOCK + t]; }
  __device__ __forceinline__ uint64_t &TH(int v) const { return th[v * PTM_BLOCK + t]; }
  __device__ __forceinline__ uint16_t &U(int v) const { return used[v * PTM_BLOCK + t]; }
  __device__ __forceinline__ uint32_t &CODE(int w) const { return code[w * PTM_BLOCK + t]; }
};

#define PTM_CODE_WORDS 9       // 71 nibbles: labels 3..73 of the longest code (labels 1, 2 are fixed)
constexpr int SCRATCH_WORDS = 28 + 42 + PTM_CODE_WORDS + 12 + 7;   // 32-bit words per k_hulls thread

// -------------------------------------------------------------- small helpers
__device__ __forceinline__ int nib(uint64_t x, int i) { return (int)((x >> (4 * i)) & 15); }
__device__ __forceinline__ uint64_t setnib(uint64_t x, int i, int v) {
  return (x & ~(15ull << (4 * i))) | ((uint64_t)v << (4 * i));
}

__device__ __forceinline__ int img_pack(int a, int b, int c) {
  return ((a + 128) << 16) | ((b + 128) << 8) | (c + 128);
}
// Packed wrap of an atom the binning excludes (non-finite coordinate, or more
// than PTM_FAR_PERIODS periods from the cell): image (-128, -128, -128), which
// no valid atom packs to.
#define PTM_FAR_PERIODS 100.f
#define PTM_EXCLUDED 0
__device__ __forceinline__ void img_unpack(int p, int &a, int &b, int &c) {
  a = ((p >> 16) & 255) - 128; b = ((p >> 8) & 255) - 128; c = (p & 255) - 128;
}

// Shift n.H in FP64 of an image outside the tables (out of line: rare).
__device__ __noinline__ void shift_far(const FrameDesc &d, int a, int b, int c, double (&s)[3]) {
  for (int k = 0; k < 3; k++)
    s[k] = __dadd_rn(__dadd_rn(__dmul_rn((double)a, d.H[k]), __dmul_rn((double)b, d.H[3 + k])),
                     __dmul_rn((double)c, d.H[6 + k]));
}

// Shift of lattice image n, rounded from FP64 exactly as the contract states.
__device__ __forceinline__ void shift_f32(const FrameDesc &d, int a, int b, int c, float &sx, float &sy,
                                          float &sz, float &lx, float &ly, float &lz) {
  if (a >= -2 && a <= 2 && b >= -2 && b <= 2 && c >= -2 && c <= 2) {
    int i = (a + 2) * 25 + (b + 2) * 5 + (c + 2);
    const ShiftTables &t = *d.tab;
    sx = t.s32[i][0]; sy = t.s32[i][1]; sz = t.s32[i][2];
    lx = t.slo[i][0]; ly = t.slo[i][1]; lz = t.slo[i][2];
  } else {
    double s[3];
    shift_far(d, a, b, c, s);
    sx = (float)s[0]; sy = (float)s[1]; sz = (float)s[2];
    lx = (float)(s[0] - (double)sx); ly = (float)(s[1] - (double)sy); lz = (float)(s[2] - (double)sz);
  }
}

__device__ __forceinline__ void shift_f64(const FrameDesc &d, int a, int b, int c, double &sx, double &sy,
                                          double &sz) {
  if (a >= -2 && a <= 2 && b >= -2 && b <= 2 && c >= -2 && c <= 2) {
    int i = (a + 2) * 25 + (b + 2) * 5 + (c + 2);
    const ShiftTables &t = *d.tab;
    sx = t.s64[i][0]; sy = t.s64[i][1]; sz = t.s64[i][2];
  } else {
    double s[3];
    shift_far(d, a, b, c, s);
    sx = s[0]; sy = s[1]; sz = s[2];
  }
}

// Error-free sum (Knuth): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// --------------------------------------------------- exact orientation + SoS
// orient(a,b,c,p) = det[b-a; c-a; p-a] on the quantised integers.  |q| <= 2^19,
// so differences fit 21 bits, cross products 42 bits and the determinant
// |.| <= 3 * 2^61 < 2^63: exact in 64-bit integers.
__device__ __forceinline__ long long orient_raw(int ax, int ay, int az, int bx, int by, int bz, int cx,
                                                int cy, int cz, int px, int py, int pz) {
  int ux = bx - ax, uy = by - ay, uz = bz - az;
  int vx = cx - ax, vy = cy - ay, vz = cz - az;
  int wx = px - ax, wy = py - ay, wz = pz - az;
  long long nx = (long long)uy * vz - (long long)uz * vy;
  long long ny = (long long)uz * vx - (long long)ux * vz;
  long long nz = (long long)ux * vy - (long long)uy * vx;
  return nx * wx + ny * wy + nz * wz;
}

// Entry (r, c) of the matrix [[q_r, 1]] for sorted row r of the four points.
__device__ __forceinline__ long long sos_entry(const Scratch &sm, const int *pt, int r, int c) {
  return c == 3 ? 1ll : (long long)sm.QI(pt[r], c);
}

// Simulation of Simplicity (Edelsbrunner & Muecke): coordinate c of the point of
// neighbour rank r is perturbed by eps^(2^(3r + c)).  With the rows sorted by
// rank, the expansion terms come in one fixed order (tables.py); the first term
// with a nonzero minor decides.  Returns the sign of orient (never 0).
__device__ __noinline__ int orient_sos_slow(const Scratch &sm, int a, int b, int c, int p) {
  int pt[4] = {a, b, c, p};
  int parity = 0;
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 3 - i; j++)
      if (pt[j] > pt[j + 1]) { int t = pt[j]; pt[j] = pt[j + 1]; pt[j + 1] = t; parity ^= 1; }
  for (int t = 0; t < PTM_SOS_NTERMS; t++) {
    int code = ptm_sos_terms[t];
    int kr = code & 15, kc = (code >> 4) & 15, neg = (code >> 8) & 1;
    int rows[3], cols[3], m = 0, mc = 0;
    for (int r = 0; r < 4; r++) if (kr >> r & 1) rows[m++] = r;
    for (int cc = 0; cc < 4; cc++) if (kc >> cc & 1) cols[mc++] = cc;
    long long v;
    if (m == 0) {
      v = 1;
    } else if (m == 1) {
      v = sos_entry(sm, pt, rows[0], cols[0]);
    } else if (m == 2) {
      v = sos_entry(sm, pt, rows[0], cols[0]) * sos_entry(sm, pt, rows[1], cols[1]) -
          sos_entry(sm, pt, rows[0], cols[1]) * sos_entry(sm, pt, rows[1], cols[0]);
    } else {
      long long e[3][3];
      for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) e[i][j] = sos_entry(sm, pt, rows[i], cols[j]);
      v = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
          e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
    }
    if (v == 0) continue;
    int s = (v > 0 ? 1 : -1) * (neg ? -1 : 1);      // sign of det of the perturbed sorted matrix
    if (parity) s = -s;                              // back to argument order
    return -s;                                       // orient = -det[[p, 1]]
  }
  return 1;   // unreachable: the last terms have minor 1
}

// FP32 filter for orient on the quantised integers.  The coordinates are exact
// floats (|q| <= 2^19), so are the differences (<= 2^20).  Each product of the
// cross product rounds by <= 2^16 and the fused difference by <= 2^17, so each
// normal component is within 2^18 of exact; the fused dot product then adds at
// most 2^37 + 3 * 2^38 (propagated) + 2^38 + 2^39 (roundings) = 13 * 2^37 < 2^41.
// |det| > 2^42 therefore fixes the sign; otherwise 0 ("decide exactly").
__device__ __forceinline__ int orient_filter(float ax, float ay, float az, float bx, float by, float bz, float cx,
                                             float cy, float cz, float px, float py, float pz) {
  const float ux = bx - ax, uy = by - ay, uz = bz - az;
  const float vx = cx - ax, vy = cy - ay, vz = cz - az;
  const float wx = px - ax, wy = py - ay, wz = pz - az;
  const float nx = fmaf(uy, vz, -(uz * vy));
  const float ny = fmaf(uz, vx, -(ux * vz));
  const float nz = fmaf(ux, vy, -(uy * vx));
  const float det = fmaf(nx, wx, fmaf(ny, wy, nz * wz));
  return det > 0x1p42f ? 1 : (det < -0x1p42f ? -1 : 0);
}

__device__ __noinline__ int orient_exact_sos(const Scratch &sm, int a, int b, int c, int p, const FrameDesc &d) {
  long long o = orient_raw(sm.QI(a, 0), sm.QI(a, 1), sm.QI(a, 2), sm.QI(b, 0), sm.QI(b, 1), sm.QI(b, 2),
                           sm.QI(c, 0), sm.QI(c, 1), sm.QI(c, 2), sm.QI(p, 0), sm.QI(p, 1), sm.QI(p, 2));
  if (o > 0) return 1;
  if (o < 0) return -1;
  count(d, C_SOS);
  return orient_sos_slow(sm, a, b, c, p);
}

// Orientation of neighbours a, b, c, p with the SoS tie rule; never 0.
__device__ __forceinline__ int orient_sos(const Scratch &sm, int a, int b, int c, int p, float px, float py,
                                          float pz, const FrameDesc &d) {
  const int s = orient_filter(sm.Q(a, 0), sm.Q(a, 1), sm.Q(a, 2), sm.Q(b, 0), sm.Q(b, 1), sm.Q(b, 2), sm.Q(c, 0),
                              sm.Q(c, 1), sm.Q(c, 2), px, py, pz);
  return s ? s : orient_exact_sos(sm, a, b, c, p, d);
}

// ------------------------------------------------------------ incremental hull
__device__ __forceinline__ uint16_t fpack(int a, int b, int c) { return (uint16_t)(a | (b << 4) | (c << 8)); }

// Tetrahedron on points 0..3, facets counter-clockwise seen from outside.
__device__ __forceinline__ int hull_init(const Scratch &sm, const FrameDesc &d) {
  int o = orient_sos(sm, 0, 1, 2, 3, sm.Q(3, 0), sm.Q(3, 1), sm.Q(3, 2), d);
  if (o < 0) {
    sm.F(0) = fpack(0, 1, 2); sm.F(1) = fpack(0, 3, 1); sm.F(2) = fpack(1, 3, 2); sm.F(3) = fpack(0, 2, 3);
  } else {
    sm.F(0) = fpack(0, 2, 1); sm.F(1) = fpack(0, 3, 2); sm.F(2) = fpack(2, 3, 1); sm.F(3) = fpack(0, 1, 3);
  }
  return 4;
}

// Signs of orient(a, b, c, p) and orient(a, b, c, origin) with the FP32 filter
// of orient_filter; both share the facet normal n = (b - a) x (c - a), and
// orient(a, b, c, origin) = -n . a (|a| <= 2^19, inside the same error bound).
// A sign of 0 means "decide exactly".
__device__ __forceinline__ void orient_pair_filter(float ax, float ay, float az, float bx, float by, float bz,
                                                   float cx, float cy, float cz, float px, float py, float pz,
                                                   int &sp, int &sc) {
  const float ux = bx - ax, uy = by - ay, uz = bz - az;
  const float vx = cx - ax, vy = cy - ay, vz = cz - az;
  const float nx = fmaf(uy, vz, -(uz * vy));
  const float ny = fmaf(uz, vx, -(ux * vz));
  const float nz = fmaf(ux, vy, -(uy * vx));
  const float dp = fmaf(nx, px - ax, fmaf(ny, py - ay, nz * (pz - az)));
  const float dc = -fmaf(nx, ax, fmaf(ny, ay, nz * az));
  sp = dp > 0x1p42f ? 1 : (dp < -0x1p42f ? -1 : 0);
  sc = dc > 0x1p42f ? 1 : (dc < -0x1p42f ? -1 : 0);
}

// Exact signs for the facets the FP32 filter left open: bit f of `openp` asks
// for orient(a, b, c, p) (SoS when exactly 0; a positive sign sets bit f of
// vis), bit f of `openc` for orient(a, b, c, origin) (exact, no SoS: zero
// clears `inside`).  One normal n = (b - a) x (c - a) in 64-bit integers serves
// both: orient(a, b, c, x) = n . (x - a).  The lanes of `wmask` take one open
// facet each per step and step together, so the 64-bit arithmetic runs once
// per step for the warp, with few values live (the filter loop has finished).
__device__ __forceinline__ void hull_exact(const Scratch &sm, int p, uint32_t openp, uint32_t openc, unsigned wmask,
                                           uint32_t &vis, bool &inside, const FrameDesc &d) {
  uint32_t open = openp | openc;
  while (__any_sync(wmask, open != 0)) {
    if (!open) continue;
    const int f = __ffs(open) - 1;
    open &= open - 1;
    const int v = sm.F(f);
    const int a = v & 15, b = (v >> 4) & 15, c = (v >> 8) & 15;
    const int ax = sm.QI(a, 0), ay = sm.QI(a, 1), az = sm.QI(a, 2);
    const int ux = sm.QI(b, 0) - ax, uy = sm.QI(b, 1) - ay, uz = sm.QI(b, 2) - az;
    const int vx = sm.QI(c, 0) - ax, vy = sm.QI(c, 1) - ay, vz = sm.QI(c, 2) - az;
    const long long nx = (long long)uy * vz - (long long)uz * vy;
    const long long ny = (long long)uz * vx - (long long)ux * vz;
    const long long nz = (long long)ux * vy - (long long)uy * vx;
    if (openp >> f & 1) {
      const long long o = nx * (sm.QI(p, 0) - ax) + ny * (sm.QI(p, 1) - ay) + nz * (sm.QI(p, 2) - az);
      int sp = (o > 0) - (o < 0);
      if (!sp) {
        count(d, C_SOS);
        sp = orient_sos_slow(sm, a, b, c, p);
      }
      if (sp > 0) vis |= 1u << f;
    }
    if (openc >> f & 1) inside &= nx * ax + ny * ay + nz * az > 0;   // orient(a, b, c, origin) = -n . a < 0
  }
}

// Facets of the current hull visible from point p (bit f set), and whether the
// centre lies strictly inside the current hull (exact, no SoS: zero rejects),
// computed only when `centre` is asked for.  Both use one normal per facet.
// `wmask`: the lanes of the warp that call this together.
__device__ uint32_t hull_visibility(const Scratch &sm, int nf, int p, bool centre, bool &centre_in, unsigned wmask,
                                    const FrameDesc &d) {
  uint32_t vis = 0, openp = 0, openc = 0;
  bool inside = true;
  const float px = sm.Q(p, 0), py = sm.Q(p, 1), pz = sm.Q(p, 2);
#pragma unroll 2
  for (int f = 0; f < nf; f++) {
    const int v = sm.F(f);
    const int a = v & 15, b = (v >> 4) & 15, c = (v >> 8) & 15;
    int sp, sc;
    orient_pair_filter(sm.Q(a, 0), sm.Q(a, 1), sm.Q(a, 2), sm.Q(b, 0), sm.Q(b, 1), sm.Q(b, 2), sm.Q(c, 0),
                       sm.Q(c, 1), sm.Q(c, 2), px, py, pz, sp, sc);
    if (sp > 0) vis |= 1u << f;
    if (!sp) openp |= 1u << f;
    if (!sc) openc |= 1u << f;
    inside &= sc <= 0;
  }
  if (!centre || !inside) openc = 0;          // the centre's answer is already known
  hull_exact(sm, p, openp, openc, wmask, vis, inside, d);
  centre_in = centre && inside;
  return vis;
}

// Centre strictly inside the current hull (for the last snapshot, where no
// further point is inserted).
__device__ bool hull_centre_inside(const Scratch &sm, int nf, unsigned wmask, const FrameDesc &d) {
  bool inside = true;
  uint32_t openc = 0;
#pragma unroll 1
  for (int f = 0; f < nf; f++) {
    const int v = sm.F(f);
    const int a = v & 15, b = (v >> 4) & 15, c = (v >> 8) & 15;
    int sp, sc;
    orient_pair_filter(sm.Q(a, 0), sm.Q(a, 1), sm.Q(a, 2), sm.Q(b, 0), sm.Q(b, 1), sm.Q(b, 2), sm.Q(c, 0),
                       sm.Q(c, 1), sm.Q(c, 2), 0.f, 0.f, 0.f, sp, sc);
    if (!sc) openc |= 1u << f;
    inside &= sc <= 0;
  }
  if (!inside) openc = 0;
  uint32_t vis = 0;
  hull_exact(sm, 0, 0, openc, wmask, vis, inside, d);
  return inside;
}

// Insert point p given its visible facets (vis != 0): remove them and fan the
// horizon to p.  Returns the new facet count, or -1 on an internal error.
__device__ int hull_apply(const Scratch &sm, int nf, uint32_t vis, int p, const FrameDesc &d) {
  // edge rows of the vertices of the visible facets only (no other row is read)
  uint32_t verts = 0;
  for (uint32_t m = vis; m; m &= m - 1) {
    const int v = sm.F(__ffs(m) - 1);
    verts |= (1u << (v & 15)) | (1u << ((v >> 4) & 15)) | (1u << ((v >> 8) & 15));
  }
  for (uint32_t m = verts; m; m &= m - 1) sm.U(__ffs(m) - 1) = 0;
  for (uint32_t m = vis; m; m &= m - 1) {
    int v = sm.F(__ffs(m) - 1);
    int a = v & 15, b = (v >> 4) & 15, c = (v >> 8) & 15;
    sm.U(a) |= 1 << b; sm.U(b) |= 1 << c; sm.U(c) |= 1 << a;
  }
  int n2 = 0;
  for (int f = 0; f < nf; f++)
    if (!(vis >> f & 1)) sm.F(n2++) = sm.F(f);
  int added = 0;
  for (uint32_t mu = verts; mu; mu &= mu - 1) {      // rows in increasing vertex order
    const int u = __ffs(mu) - 1;
    uint32_t row = sm.U(u);
    while (row) {
      int v = __ffs(row) - 1;
      row &= row - 1;
      if (!(sm.U(v) >> u & 1)) {               // horizon edge u -> v
        if (n2 < 24) sm.F(n2) = fpack(u, v, p);
        n2++;
        added++;
      }
    }
  }
  // a triangulated disk of F visible facets with I interior vertices has
  // F + 2 - 2I boundary edges; swallowed vertices simply leave the facet list
  if (added < 3 || added > __popc(vis) + 2 || ((added - __popc(vis)) & 1) || n2 > 24) {
    count(d, C_INTERNAL);
    return -1;
  }
  return n2;
}

// ------------------------------------------------------- Weinberg code
// Walk from u -> v over the K-vertex hull (rules in tables.py), writing the
// code (labels 3.. as nibbles; every walk starts with labels 1, 2) to the CODE
// rows and the first-visit labelling to `labels`.  False on an internal error.
__device__ bool weinberg_walk(const Scratch &sm, int K, int u, int v, uint64_t &labels, const FrameDesc &d) {
  const int LEN = 2 * (3 * K - 6) + 1;
  uint64_t lab = 0;
#pragma unroll
  for (int x = 0; x < PTM_KNN; x++) sm.U(x) = 0;
  int next = 1;
  uint32_t wbuf = 0;
  auto emit = [&](int s, int L) {
    const int n = s - 2;
    wbuf |= (uint32_t)L << (4 * (n & 7));
    if ((n & 7) == 7 || s == LEN - 1) { sm.CODE(n >> 3) = wbuf; wbuf = 0; }
  };
  lab = setnib(lab, u, next++);
  sm.U(u) |= 1 << v;
  bool fresh = true;
  lab = setnib(lab, v, next++);
  int s = 2;
  for (; s < LEN; s++) {
    const uint64_t tv = sm.TH(v);
    const uint32_t uv = sm.U(v);
    int w = nib(tv, u);                              // next edge counter-clockwise
    if (!fresh) {
      if (!(uv >> u & 1)) {
        w = u;                                       // old vertex, new edge: walk back
      } else {
        int guard = 0;                               // first unused edge after arrival
        while (w != u && (uv >> w & 1) && guard++ < 16) w = nib(tv, w);
        if (w == u || guard > 16) break;
      }
    }
    if (w >= K) { count(d, C_INTERNAL); return false; }
    sm.U(v) = (uint16_t)(uv | (1u << w));
    u = v;
    v = w;
    int L = nib(lab, v);
    fresh = (L == 0);
    if (fresh) { L = next++; lab = setnib(lab, v, L); }
    emit(s, L);
  }
  if (s != LEN) { count(d, C_INTERNAL); return false; }
  labels = lab;
  return true;
}

// Weinberg code of the current K-vertex hull for the table lookup.  Every
// directed edge u->v gets the key (deg u, deg v, deg w1, deg w2) with (u, v, w1)
// and (v, u, w2) the two facets on the edge, continued (for edges tied on it)
// by the degrees of the third vertices of the facets across their four outer
// edges; the walk starts from the first edge with the largest key (definition
// in tables.py, whose tables hold the code of every such start).  Returns the
// labelling (nibble t = label of neighbour t) and the code hash; false on an
// internal error.  Every lane walks once, so a warp's walks run together.
__device__ bool canonical(const Scratch &sm, int K, int nf, uint64_t &labels, uint64_t &hash,
                          const FrameDesc &d) {
  uint64_t deg = 0;
#pragma unroll
  for (int x = 0; x < PTM_KNN; x++) sm.TH(x) = ~0ull;
  for (int f = 0; f < nf; f++) {
    int v = sm.F(f);
    int a = v & 15, b = (v >> 4) & 15, c = (v >> 8) & 15;
    sm.TH(a) = setnib(sm.TH(a), b, c);
    sm.TH(b) = setnib(sm.TH(b), c, a);
    sm.TH(c) = setnib(sm.TH(c), a, b);
    deg += (1ull << (4 * a)) + (1ull << (4 * b)) + (1ull << (4 * c));
  }
  // keys of the directed edges (a->b, b->c, c->a of every facet); keep the maximum
  uint32_t top = 0;
  uint64_t m0 = 0;          // edge ids 0..63 (id = 3 f + corner)
  uint32_t m1 = 0;          // edge ids 64..71
  for (int f = 0; f < nf; f++) {
    const int v = sm.F(f);
    const int p0 = v & 15, p1 = (v >> 4) & 15, p2 = (v >> 8) & 15;
    const int dg0 = nib(deg, p0), dg1 = nib(deg, p1), dg2 = nib(deg, p2);
#pragma unroll
    for (int e = 0; e < 3; e++) {
      const int x = e == 0 ? p0 : (e == 1 ? p1 : p2);      // edge x -> y, third vertex z
      const int y = e == 0 ? p1 : (e == 1 ? p2 : p0);
      const int dx = e == 0 ? dg0 : (e == 1 ? dg1 : dg2);
      const int dy = e == 0 ? dg1 : (e == 1 ? dg2 : dg0);
      const int dz = e == 0 ? dg2 : (e == 1 ? dg0 : dg1);
      const int w2 = nib(sm.TH(y), x);
      const uint32_t key = (uint32_t)((dx << 12) | (dy << 8) | (dz << 4) | nib(deg, w2));
      const int id = 3 * f + e;
      if (key > top) { top = key; m0 = 0; m1 = 0; }
      if (key == top) { if (id < 64) m0 |= 1ull << id; else m1 |= 1u << (id - 64); }
    }
  }
  // K = 12 with every degree 5 is the icosahedron, K = 6 with every degree 4 the
  // octahedron: every directed edge has the same key
  const bool transitive = (K == 12 && top == 0x5555u) || (K == 6 && top == 0x4444u);
  // edges tied on the degrees of the edge's two facets: the key continues with
  // the degrees of the third vertices of the facets across their outer edges
  if (!transitive && __popcll((long long)m0) + __popc(m1) > 1) {
    uint32_t etop = 0;
    uint64_t n0 = 0;
    uint32_t n1 = 0;
    auto consider = [&](int id) {
      const int v = sm.F(id / 3), e = id % 3;
      const int p0 = v & 15, p1 = (v >> 4) & 15, p2 = (v >> 8) & 15;
      const int x = e == 0 ? p0 : (e == 1 ? p1 : p2);      // edge x -> y, third vertex z
      const int y = e == 0 ? p1 : (e == 1 ? p2 : p0);
      const int z = e == 0 ? p2 : (e == 1 ? p0 : p1);
      const int w = nib(sm.TH(y), x);
      const uint32_t ext = (uint32_t)((nib(deg, nib(sm.TH(z), y)) << 12) | (nib(deg, nib(sm.TH(x), z)) << 8) |
                                      (nib(deg, nib(sm.TH(w), x)) << 4) | nib(deg, nib(sm.TH(y), w)));
      if (ext > etop) { etop = ext; n0 = 0; n1 = 0; }
      if (ext == etop) { if (id < 64) n0 |= 1ull << id; else n1 |= 1u << (id - 64); }
    };
    for (uint64_t mm = m0; mm; mm &= mm - 1) consider(__ffsll((long long)mm) - 1);
    for (uint32_t mm = m1; mm; mm &= mm - 1) consider(64 + __ffs(mm) - 1);
    m0 = n0;
    m1 = n1;
  }
  // one walk, from the first start edge with the largest key: the tables hold
  // the code of every such start of every template triangulation
  if (!(m0 | m1)) return false;
  const int id = m0 ? __ffsll((long long)m0) - 1 : 64 + __ffs(m1) - 1;
  {
    const int v = sm.F(id / 3), e = id % 3;
    const int p0 = v & 15, p1 = (v >> 4) & 15, p2 = (v >> 8) & 15;
    const int su = e == 0 ? p0 : (e == 1 ? p1 : p2);
    const int sv = e == 0 ? p1 : (e == 1 ? p2 : p0);
    if (!weinberg_walk(sm, K, su, sv, labels, d)) return false;
  }
  // hash of the packed code (labels 3..LEN); words past its end count as zero,
  // as the generator packs them
  const int LEN = 2 * (3 * K - 6) + 1;
  uint64_t h = PTM_HASH_INIT;
#pragma unroll
  for (int w = 0; w < PTM_CODE_WORDS; w++) h = (h ^ (uint64_t)(w * 8 < LEN - 2 ? sm.CODE(w) : 0u)) * PTM_HASH_MUL;
  hash = h;
  return true;
}

// ------------------------------------------------------------------- QCP
// Horn's 4x4 matrix from S_ab = sum_i w_ia v_ib (template w rotated onto data v),
// characteristic polynomial P(l) = l^4 + c2 l^2 + c1 l + c0 with c2 = -2|S|^2,
// c1 = -8 det S, c0 = det K (Theobald 2005), largest root by Newton from the
// upper bound sqrt(Gv Gw) (Cauchy-Schwarz).
template <typename T>
struct Qcp {
  T K[4][4];
  T lam, dP;
  int iters;
};

template <typename T>
__device__ __forceinline__ void horn_matrix(const T S[3][3], T K[4][4]) {
  K[0][0] = S[0][0] + S[1][1] + S[2][2];
  K[0][1] = S[1][2] - S[2][1];
  K[0][2] = S[2][0] - S[0][2];
  K[0][3] = S[0][1] - S[1][0];
  K[1][1] = S[0][0] - S[1][1] - S[2][2];
  K[1][2] = S[0][1] + S[1][0];
  K[1][3] = S[2][0] + S[0][2];
  K[2][2] = -S[0][0] + S[1][1] - S[2][2];
  K[2][3] = S[1][2] + S[2][1];
  K[3][3] = -S[0][0] - S[1][1] + S[2][2];
  K[1][0] = K[0][1]; K[2][0] = K[0][2]; K[3][0] = K[0][3];
  K[2][1] = K[1][2]; K[3][1] = K[1][3]; K[3][2] = K[2][3];
}

template <typename T>
__device__ __forceinline__ T det4(const T a[4][4]) {
  // Laplace expansion over the 2x2 minors of rows 0-1 and rows 2-3
  T s0 = a[0][0] * a[1][1] - a[1][0] * a[0][1];
  T s1 = a[0][0] * a[1][2] - a[1][0] * a[0][2];
  T s2 = a[0][0] * a[1][3] - a[1][0] * a[0][3];
  T s3 = a[0][1] * a[1][2] - a[1][1] * a[0][2];
  T s4 = a[0][1] * a[1][3] - a[1][1] * a[0][3];
  T s5 = a[0][2] * a[1][3] - a[1][2] * a[0][3];
  T c5 = a[2][2] * a[3][3] - a[3][2] * a[2][3];
  T c4 = a[2][1] * a[3][3] - a[3][1] * a[2][3];
  T c3 = a[2][1] * a[3][2] - a[3][1] * a[2][2];
  T c2 = a[2][0] * a[3][3] - a[3][0] * a[2][3];
  T c1 = a[2][0] * a[3][2] - a[3][0] * a[2][2];
  T c0 = a[2][0] * a[3][1] - a[3][0] * a[2][1];
  return s0 * c5 - s1 * c4 + s2 * c3 + s3 * c2 - s4 * c1 + s5 * c0;
}

template <typename T>
__device__ __forceinline__ T det3(const T m[3][3]) {
  return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
         m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

template <typename T>
__device__ void qcp_solve(const T S[3][3], T Gv, T Gw, Qcp<T> &o) {
  horn_matrix<T>(S, o.K);
  T n2 = 0;
  for (int a = 0; a < 3; a++) for (int b = 0; b < 3; b++) n2 += S[a][b] * S[a][b];
  T c2 = T(-2) * n2;
  T c1 = T(-8) * det3<T>(S);
  T c0 = det4<T>(o.K);
  T lam = sqrt(Gv * Gw);
  const T tol = sizeof(T) == 4 ? T(1e-7) : T(1e-15);
  T dP = 0;
  int it = 0;
  for (; it < 60; it++) {
    T l2 = lam * lam;
    T P = (l2 + c2) * l2 + c1 * lam + c0;
    dP = (T(4) * l2 + T(2) * c2) * lam + c1;
    if (!(dP > T(0))) break;
    T delta = P / dP;
    lam -= delta;
    if (fabs(delta) <= tol * lam) { it++; break; }
  }
  T l2 = lam * lam;
  o.dP = (T(4) * l2 + T(2) * c2) * lam + c1;
  o.lam = lam;
  o.iters = it;
}

// Unit quaternion of the largest eigenvalue: the column of adj(K - lam I) with
// the largest norm (all nonzero columns are parallel to the eigenvector).
// Cofactor (c, r) deletes row c and column r; every index is static once the
// loops are unrolled, so nothing lands in local memory.
template <typename T>
__device__ void qcp_quat(const T K[4][4], T lam, T q[4]) {
  T A[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) A[i][j] = K[i][j] - (i == j ? lam : T(0));
  T best = T(-1);
  T b0 = 1, b1 = 0, b2 = 0, b3 = 0;
#pragma unroll
  for (int c = 0; c < 4; c++) {
    T col[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
      T m[3][3];
#pragma unroll
      for (int ii = 0; ii < 3; ii++)
#pragma unroll
        for (int jj = 0; jj < 3; jj++) m[ii][jj] = A[ii + (ii >= c)][jj + (jj >= r)];
      const T v = det3<T>(m);
      col[r] = ((c + r) & 1) ? -v : v;
    }
    const T nn = col[0] * col[0] + col[1] * col[1] + col[2] * col[2] + col[3] * col[3];
    if (nn > best) { best = nn; b0 = col[0]; b1 = col[1]; b2 = col[2]; b3 = col[3]; }
  }
  if (!(best > T(0))) { q[0] = 1; q[1] = q[2] = q[3] = 0; return; }
  T inv = T(1) / sqrt(best);
  if (b0 < T(0)) inv = -inv;
  q[0] = b0 * inv; q[1] = b1 * inv; q[2] = b2 * inv; q[3] = b3 * inv;
}

template <typename T>
__device__ __forceinline__ void quat_matrix(const T q[4], T R[3][3]) {
  T w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix.
template <typename T>
__device__ void jacobi3(T a[3][3], T v[3][3]) {
  const T tol = sizeof(T) == 4 ? (T)1e-16 : (T)1e-30;
  for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) v[i][j] = (i == j) ? (T)1 : (T)0;
  for (int sweep = 0; sweep < (sizeof(T) == 4 ? 10 : 20); sweep++) {
    T off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    T dg = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (off <= tol * dg) break;
#pragma unroll
    for (int pq = 0; pq < 3; pq++) {
      int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      if (a[p][q] == (T)0) continue;
      T theta = (a[q][q] - a[p][p]) / ((T)2 * a[p][q]);
      T t = (theta >= (T)0 ? (T)1 : (T)-1) / (fabs(theta) + sqrt(theta * theta + (T)1));
      T c = rsq(t * t + (T)1), s = t * c;
      for (int k = 0; k < 3; k++) {
        T akp = a[k][p], akq = a[k][q];
        a[k][p] = c * akp - s * akq; a[k][q] = s * akp + c * akq;
      }
      for (int k = 0; k < 3; k++) {
        T apk = a[p][k], aqk = a[q][k];
        a[p][k] = c * apk - s * aqk; a[q][k] = s * apk + c * aqk;
      }
      for (int k = 0; k < 3; k++) {
        T vkp = v[k][p], vkq = v[k][q];
        v[k][p] = c * vkp - s * vkq; v[k][q] = s * vkp + c * vkq;
      }
    }
  }
}

}  // namespace ptm
