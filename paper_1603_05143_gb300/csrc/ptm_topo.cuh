// Topological neighbour ordering (Sec. 3, Eq. 5): for every atom, its 18
// nearest images (the distance contract of the Euclidean path), the area of the
// face its Voronoi cell shares with each of them (the cell taken among those 18,
// as Sec. 9 does with the Delaunay triangulation of the centre and its 18
// nearest), and the order "larger face first, then nearer".  The first 14 in
// that order replace the 14 nearest for the rest of the method.
//
// Face area of neighbour j: the bisector plane x.v_j = |v_j|^2 / 2, clipped by
// every other neighbour's half-space x.v_i <= |v_i|^2 / 2 (one half-plane at a
// time, in plane coordinates), then the shoelace formula; 0 when nothing is
// left.  Floating point cannot reproduce exact ties between equal faces (the 12
// faces of a perfect fcc cell), so areas that follow each other in descending
// order within TOPO_BAND x the mean squared distance form one group, ordered by
// the Euclidean rank (distance, atom id, image).  FP32 areas decide unless a
// gap lies within TOPO_GUARD of the band edge; then the atom's areas are
// recomputed in FP64 from FP64 neighbour vectors, by a second kernel over just
// those atoms.

namespace ptm {

#define PTM_TOPO_N 18
#define PTM_TOPO_BAND 1e-3
#define PTM_TOPO_GUARD 2e-5
#define PTM_TOPO_VMAX 24       // FP64 polygon buffer: 4 + 17 clips add at most 21 vertices
// FP32 pass: polygons of up to 12 vertices in shared memory (the largest polygon met
// while clipping an atom's 18 faces had 11 vertices in 6,000 atoms of crystals and
// liquid); an atom whose clipping outgrows it is left to the FP64 pass
#define PTM_TOPO_VMAX32 12
// 32-bit words per thread: neighbour ids and images, FP32 vectors, two polygon buffers
#define PTM_TOPO_WORDS (2 * PTM_TOPO_N + 3 * PTM_TOPO_N + 2 * 2 * PTM_TOPO_VMAX32)
// Resident blocks per SM that shared memory allows: 6 for the FP32 pass (138
// words x 64 threads), 4 for the FP64 pass (its polygon buffers).  Stating them
// lets the compiler give each thread the registers that occupancy leaves free
// (94-127 instead of 56-96, and no spills).
#define PTM_TOPO_BLOCKS_PER_SM 6
#define PTM_TOPO64_BLOCKS_PER_SM 4

// Area of the Voronoi face of neighbour j among the m vectors V(i, c); P and Q
// are polygon buffers of 2 x vmax values, element e at P[e * st].  A clip that
// would leave more than vmax vertices sets `over` (the polygon keeps its first
// vmax vertices).
template <typename T, typename Vec>
__device__ T topo_face_area(int m, int j, T R, Vec V, T *P, T *Q, int st, int vmax, bool &over) {
  const T n0 = V(j, 0), n1 = V(j, 1), n2 = V(j, 2);
  const T nn = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
  const T u0 = n0 / nn, u1 = n1 / nn, u2 = n2 / nn;
  // e1 = u x a with a the axis least aligned with u, e2 = u x e1
  const bool ax = fabs(u0) < (T)0.6;
  const T a0 = ax ? (T)1 : (T)0, a1 = ax ? (T)0 : (T)1;
  T e10 = u1 * (T)0 - u2 * a1, e11 = u2 * a0 - u0 * (T)0, e12 = u0 * a1 - u1 * a0;
  const T l1 = sqrt(e10 * e10 + e11 * e11 + e12 * e12);
  e10 /= l1; e11 /= l1; e12 /= l1;
  const T e20 = u1 * e12 - u2 * e11, e21 = u2 * e10 - u0 * e12, e22 = u0 * e11 - u1 * e10;
  const T p0 = n0 / 2, p1 = n1 / 2, p2 = n2 / 2;
  // a convex polygon gains at most one vertex per clip (4 + 17 < PTM_TOPO_VMAX);
  // rounding on a nearly degenerate polygon could emit more, so writes stop at
  // the buffer's end (the polygon then has next to no area either way)
  T *cur = P, *nxt = Q;
  int np = 4;
  cur[0] = -R; cur[st] = -R; cur[2 * st] = R; cur[3 * st] = -R;
  cur[4 * st] = R; cur[5 * st] = R; cur[6 * st] = -R; cur[7 * st] = R;
  for (int i = 0; i < m && np > 0; i++) {
    if (i == j) continue;
    const T w0 = V(i, 0), w1 = V(i, 1), w2 = V(i, 2);
    const T A = w0 * e10 + w1 * e11 + w2 * e12, B = w0 * e20 + w1 * e21 + w2 * e22;
    const T C = (w0 * w0 + w1 * w1 + w2 * w2) / 2 - (w0 * p0 + w1 * p1 + w2 * p2);
    int nq = 0;
    for (int k = 0; k < np; k++) {
      const int k1 = k + 1 == np ? 0 : k + 1;
      const T xs = cur[2 * k * st], xt = cur[(2 * k + 1) * st], ys = cur[2 * k1 * st], yt = cur[(2 * k1 + 1) * st];
      const T fx = A * xs + B * xt - C, fy = A * ys + B * yt - C;
      if (fx <= 0) {
        if (nq < vmax) { nxt[2 * nq * st] = xs; nxt[(2 * nq + 1) * st] = xt; }
        nq++;
      }
      if ((fx < 0 && fy > 0) || (fx > 0 && fy < 0)) {
        const T tt = fx / (fx - fy);
        if (nq < vmax) { nxt[2 * nq * st] = xs + tt * (ys - xs); nxt[(2 * nq + 1) * st] = xt + tt * (yt - xt); }
        nq++;
      }
    }
    over |= nq > vmax;
    np = min(nq, vmax);
    T *tmp = cur; cur = nxt; nxt = tmp;
  }
  T s2 = 0;
  for (int k = 0; k < np; k++) {
    const int k1 = k + 1 == np ? 0 : k + 1;
    s2 += cur[2 * k * st] * cur[(2 * k1 + 1) * st] - cur[2 * k1 * st] * cur[(2 * k + 1) * st];
  }
  return fabs(s2) / 2;
}

// Order o[0..m) of neighbour ranks by (area descending, rank ascending), then
// group by the band and order each group by rank.  Returns the faces (bit =
// neighbour rank) on either side of a gap between consecutive areas that lies
// within the guard of the band edge; 0 when every gap is clear of it.
template <typename T>
__device__ uint32_t topo_order(int m, const T *area, T mean2, int *o) {
  for (int k = 0; k < m; k++) o[k] = k;
  for (int k = 1; k < m; k++) {                       // insertion sort, stable in rank
    const int x = o[k];
    int p = k;
    while (p > 0 && area[o[p - 1]] < area[x]) { o[p] = o[p - 1]; p--; }
    o[p] = x;
  }
  const T band = (T)PTM_TOPO_BAND * mean2, guard = (T)PTM_TOPO_GUARD * mean2;
  uint32_t near = 0;
  int g0 = 0;
  for (int k = 1; k <= m; k++) {
    bool split = k == m;
    if (k < m) {
      const T gap = area[o[k - 1]] - area[o[k]];
      if (fabs(gap - band) <= guard) near |= (1u << o[k - 1]) | (1u << o[k]);
      split = gap > band;
    }
    if (split) {                                      // group o[g0..k): order by rank
      for (int a = g0 + 1; a < k; a++) {
        const int x = o[a];
        int p = a;
        while (p > g0 && o[p - 1] > x) { o[p] = o[p - 1]; p--; }
        o[p] = x;
      }
      g0 = k;
    }
  }
  return near;
}

// kNN slots in the topological scratch: rows J (sorted index) and IMG (packed
// image), then (while a run is ordered) the atom id and FP64 key in the rows of
// the FP32 vectors (3 x 18 rows), which are written only after the kNN.
typedef SmemKnnRows<PTM_TOPO_N, PTM_BLOCK> TopoKnnRows;
static_assert(TopoKnnRows::kRows <= 5 * PTM_TOPO_N, "kNN rows must fit the neighbour and vector rows");

// What the FP32 pass leaves for the FP64 pass about a listed atom: its 18
// neighbours, their FP32 face areas and the faces to recompute in FP64 (bit =
// neighbour rank: the two faces of every gap at the band edge, or all).
struct TopoSide {
  int2 nb[PTM_TOPO_N];
  float area[PTM_TOPO_N];
  uint32_t faces;
  uint32_t pad;
};

// One atom, FP32 areas.  An atom with an area gap at the band edge (or a
// polygon larger than the FP32 buffers) is appended to `list` for the FP64 pass
// instead of being decided here, so that no warp waits on one lane's FP64 work;
// the first cap_side listed atoms leave their neighbours, areas and uncertain
// faces in `side`.
template <bool F64>
__device__ void topo_atom(const FrameDesc &d, int s, int *tsm, int2 *__restrict__ out, int *list, int *list_count,
                          TopoSide *side, int cap_side) {
  typedef typename RT<F64>::T TI;
  const int t = threadIdx.x;
  auto J = [&](int k) -> int & { return tsm[k * PTM_BLOCK + t]; };
  auto IMG = [&](int k) -> int & { return tsm[(PTM_TOPO_N + k) * PTM_BLOCK + t]; };
  auto VF = [&](int k, int c) -> float & { return ((float *)tsm)[(2 * PTM_TOPO_N + 3 * k + c) * PTM_BLOCK + t]; };
  const int64_t n = d.n, sl = s - d.atom_offset;     // frame-local slot
  if (__ldg(d.wrapv + s) == PTM_EXCLUDED) {           // excluded by the binning: no neighbours
    for (int k = 0; k < PTM_KNN; k++) out[(int64_t)k * n + sl] = make_int2(-1, 0);
    return;
  }
  TI xi, yi, zi;
  int idi;
  load_atom<F64>(d, s, xi, yi, zi, idi);
  const int b = __ldg(d.sbin + s);
  const int bz = b % d.nb[2], byx = b / d.nb[2];
  const int by = byx % d.nb[1], bx = byx / d.nb[1];
  const bool wrapped = d.dstat[0] != 0;
  int wix = 0, wiy = 0, wiz = 0;
  if (wrapped) img_unpack(__ldg(d.wrapv + s), wix, wiy, wiz);

  // ---- the 18 nearest images
  int m;
  uint32_t close_runs = 0;
  if (!wrapped && knn_fast_n<F64, PTM_TOPO_N>(d, s, xi, yi, zi, bx, by, bz, TopoKnnRows{tsm, t}, close_runs)) {
    m = PTM_TOPO_N;
    if (!F64 && close_runs) count(d, C_KNN64);
  } else {
    double Ld2[PTM_TOPO_N];
    int Lid[PTM_TOPO_N], Ljs[PTM_TOPO_N], Limg[PTM_TOPO_N];
    m = knn<F64, PTM_TOPO_N>(d, s, xi, yi, zi, bx, by, bz, wix, wiy, wiz, wrapped, Ld2, Lid, Ljs, Limg);
    if (m < 0) m = 0;
#pragma unroll
    for (int k = 0; k < PTM_TOPO_N; k++) { J(k) = Ljs[k]; IMG(k) = Limg[k]; }
  }
  int o[PTM_TOPO_N];
  // FP32 neighbour vectors: the difference of positions plus the image
  // shift, summed without loss (error-free sums), as the metric steps use them
  float mean2 = 0.f, dmax2 = 0.f;
  for (int k = 0; k < m; k++) {
    TI xj, yj, zj;
    int idj;
    load_atom<F64>(d, J(k), xj, yj, zj, idj);
    int a0, a1, a2;
    img_unpack(IMG(k), a0, a1, a2);
    if constexpr (F64) {
      double hx, hy, hz;
      shift_f64(d, a0, a1, a2, hx, hy, hz);
      VF(k, 0) = (float)((xj - xi) + hx); VF(k, 1) = (float)((yj - yi) + hy); VF(k, 2) = (float)((zj - zi) + hz);
    } else {
      float hx, hy, hz, lx, ly, lz, p, e1, q2, e2;
      shift_f32(d, a0, a1, a2, hx, hy, hz, lx, ly, lz);
      two_sum(xj, -xi, p, e1); two_sum(p, hx, q2, e2); VF(k, 0) = q2 + (e1 + (e2 + lx));
      two_sum(yj, -yi, p, e1); two_sum(p, hy, q2, e2); VF(k, 1) = q2 + (e1 + (e2 + ly));
      two_sum(zj, -zi, p, e1); two_sum(p, hz, q2, e2); VF(k, 2) = q2 + (e1 + (e2 + lz));
    }
    const float r2 = VF(k, 0) * VF(k, 0) + VF(k, 1) * VF(k, 1) + VF(k, 2) * VF(k, 2);
    mean2 += r2;
    dmax2 = fmaxf(dmax2, r2);
  }
  if (m > 0) {
    mean2 /= (float)m;
    const float R = 10.f * sqrtf(dmax2);
    auto vf = [&](int i, int c) -> float { return VF(i, c); };
    // polygon buffers in shared memory, one word per thread per row
    float *PB = (float *)tsm + 5 * PTM_TOPO_N * PTM_BLOCK + t;
    float *QB = PB + 2 * PTM_TOPO_VMAX32 * PTM_BLOCK;
    float area[PTM_TOPO_N];
    bool over = false;
    for (int k = 0; k < m; k++) area[k] = topo_face_area<float>(m, k, R, vf, PB, QB, PTM_BLOCK, PTM_TOPO_VMAX32, over);
    // a gap at the band edge, or a polygon larger than the buffer: the second pass decides
    const uint32_t near = topo_order<float>(m, area, mean2, o);
    if (near || over) {
      count(d, C_TOPO64);
      const int slot = atomicAdd(list_count, 1);
      list[slot] = s;
      if (slot < cap_side) {                      // what the FP64 pass reuses
        TopoSide &sd = side[slot];
        for (int k = 0; k < PTM_TOPO_N; k++) {
          sd.nb[k] = k < m ? make_int2(J(k), IMG(k)) : make_int2(-1, 0);
          sd.area[k] = k < m ? area[k] : 0.f;
        }
        sd.faces = over ? ~0u : near;
      }
    }
  }
  for (int k = 0; k < PTM_KNN; k++)
    out[(int64_t)k * n + sl] = k < m ? make_int2(J(o[k]), IMG(o[k])) : make_int2(-1, 0);
}

// FP64 pass for listed atom i (= list position), one thread: FP64 neighbour
// vectors, and in FP64 the areas of the faces the FP32 pass could not decide
// (the two faces of every gap at the band edge); the others keep their FP32
// areas, whose error (measured within 2.2e-6 of the mean squared distance) is
// far below the guard, so every gap decided from them is decided as in FP64.
// Atoms past the side buffer find their neighbours again and recompute every
// face.  Polygon buffers in shared memory, element e at P[e * PTM_BLOCK].  The
// lanes of `wmask` call this together and take their faces in step, one face
// per lane per trip, so a warp makes as many trips as its busiest lane has
// faces (not one per face index that any lane needs).
template <bool F64>
__device__ void topo_atom64(const FrameDesc &d, int s, int i, const TopoSide *side, int cap_side, double *P,
                            double *Q, int2 *__restrict__ out, unsigned wmask) {
  typedef typename RT<F64>::T TI;
  TI xi, yi, zi;
  int idi;
  load_atom<F64>(d, s, xi, yi, zi, idi);
  int jn[PTM_TOPO_N], im[PTM_TOPO_N], m = 0;
  double a64[PTM_TOPO_N];
  uint32_t faces = ~0u;
  if (i < cap_side) {
    const TopoSide &sd = side[i];
    for (int k = 0; k < PTM_TOPO_N; k++) {
      const int2 e = sd.nb[k];
      jn[k] = e.x;
      im[k] = e.y;
      a64[k] = (double)sd.area[k];
      m += e.x >= 0;
    }
    faces = sd.faces;
  } else {
    const int b = __ldg(d.sbin + s);
    const int bz = b % d.nb[2], byx = b / d.nb[2];
    const int by = byx % d.nb[1], bx = byx / d.nb[1];
    const bool wrapped = d.dstat[0] != 0;
    int wix = 0, wiy = 0, wiz = 0;
    if (wrapped) img_unpack(__ldg(d.wrapv + s), wix, wiy, wiz);
    double Ld2[PTM_TOPO_N];
    int Lid[PTM_TOPO_N];
    m = knn<F64, PTM_TOPO_N>(d, s, xi, yi, zi, bx, by, bz, wix, wiy, wiz, wrapped, Ld2, Lid, jn, im);
    if (m < 0) m = 0;
  }
  int o[PTM_TOPO_N];
  double v64[PTM_TOPO_N][3], mean64 = 0.0, dmax64 = 0.0;
  if (m > 0) {
    for (int k = 0; k < m; k++) {
      vec_fp64<F64>(d, xi, yi, zi, jn[k], im[k], v64[k][0], v64[k][1], v64[k][2]);
      const double r2 = v64[k][0] * v64[k][0] + v64[k][1] * v64[k][1] + v64[k][2] * v64[k][2];
      mean64 += r2;
      dmax64 = fmax(dmax64, r2);
    }
    mean64 /= m;
  }
  auto vd = [&](int a, int c) -> double { return v64[a][c]; };
  bool over = false;
  uint32_t todo = m > 0 ? faces & ((1u << m) - 1u) : 0u;
  while (__any_sync(wmask, todo != 0)) {
    if (!todo) continue;
    const int k = __ffs(todo) - 1;
    todo &= todo - 1;
    a64[k] = topo_face_area<double>(m, k, 10.0 * sqrt(dmax64), vd, P, Q, PTM_BLOCK, PTM_TOPO_VMAX, over);
  }
  if (m > 0) topo_order<double>(m, a64, mean64, o);
  const int64_t n = d.n, sl = s - d.atom_offset;     // frame-local slot
  for (int k = 0; k < PTM_KNN; k++) out[(int64_t)k * n + sl] = k < m ? make_int2(jn[o[k]], im[o[k]]) : make_int2(-1, 0);
}

template <bool F64>
__global__ void __launch_bounds__(PTM_BLOCK, PTM_TOPO_BLOCKS_PER_SM) k_topo(const __grid_constant__ FrameDesc d, int2 *__restrict__ out,
                                                    int *list, int *list_count, TopoSide *side, int cap_side) {
  extern __shared__ __align__(16) unsigned char tsm_raw[];
  const int64_t s = (int64_t)blockIdx.x * PTM_BLOCK + threadIdx.x;
  if (s >= d.n) return;
  topo_atom<F64>(d, (int)s, (int *)tsm_raw, out, list, list_count, side, cap_side);
}

// Second pass over the listed atoms, one thread per atom (grid-stride over the
// list: its length is read on the device).
template <bool F64>
__global__ void __launch_bounds__(PTM_BLOCK, PTM_TOPO64_BLOCKS_PER_SM) k_topo64(const __grid_constant__ FrameDesc d, int2 *__restrict__ out,
                                                      const int *list, const int *list_count, const TopoSide *side,
                                                      int cap_side) {
  extern __shared__ __align__(16) unsigned char tsm_raw[];
  double *P = (double *)tsm_raw + threadIdx.x, *Q = P + 2 * PTM_TOPO_VMAX * PTM_BLOCK;
  const int cnt = *list_count;
  for (int i0 = blockIdx.x * PTM_BLOCK + (threadIdx.x & ~31); i0 < cnt; i0 += gridDim.x * PTM_BLOCK) {
    const int i = i0 + (threadIdx.x & 31);
    const unsigned wmask = __ballot_sync(0xffffffffu, i < cnt);
    if (i < cnt) topo_atom64<F64>(d, list[i], i, side, cap_side, P, Q, out, wmask);
  }
}

// The same two passes over a batch: every slot finds its frame (frames in the
// Euclidean order have no topological buffer and are skipped); each frame's
// order lands in its own segment of the batch's buffer (FrameDesc::topo).
template <bool F64>
__global__ void __launch_bounds__(PTM_BLOCK, PTM_TOPO_BLOCKS_PER_SM)
    k_topo_batch(const FrameDesc *__restrict__ descs, const int64_t *__restrict__ atom_off, int nframes,
                 int64_t ntotal, int *list, int *list_count, TopoSide *side, int cap_side) {
  extern __shared__ __align__(16) unsigned char tsm_raw[];
  const int64_t s = (int64_t)blockIdx.x * PTM_BLOCK + threadIdx.x;
  if (s >= ntotal) return;
  const FrameDesc &d = descs[frame_of(atom_off, nframes, s)];
  if (d.ordering != PTM_ORDER_TOPOLOGICAL) return;
  topo_atom<F64>(d, (int)s, (int *)tsm_raw, const_cast<int2 *>(d.nbr), list, list_count, side, cap_side);
}

template <bool F64>
__global__ void __launch_bounds__(PTM_BLOCK, PTM_TOPO64_BLOCKS_PER_SM)
    k_topo64_batch(const FrameDesc *__restrict__ descs, const int64_t *__restrict__ atom_off, int nframes,
                   const int *list, const int *list_count, const TopoSide *side, int cap_side) {
  extern __shared__ __align__(16) unsigned char tsm_raw[];
  double *P = (double *)tsm_raw + threadIdx.x, *Q = P + 2 * PTM_TOPO_VMAX * PTM_BLOCK;
  const int cnt = *list_count;
  for (int i0 = blockIdx.x * PTM_BLOCK + (threadIdx.x & ~31); i0 < cnt; i0 += gridDim.x * PTM_BLOCK) {
    const int i = i0 + (threadIdx.x & 31);
    const unsigned wmask = __ballot_sync(0xffffffffu, i < cnt);
    if (i < cnt) {
      const int s = list[i];
      const FrameDesc &d = descs[frame_of(atom_off, nframes, s)];
      topo_atom64<F64>(d, s, i, side, cap_side, P, Q, const_cast<int2 *>(d.nbr), wmask);
    }
  }
}

// Listed atoms whose neighbours, areas and uncertain faces the FP32 pass keeps
// for the FP64 pass (a quarter of the atoms: 3.6 % were listed in the hot
// polycrystal, 2.6 % in the mixed-phase frame, up to 15 % in cold crystals; the
// rest find their neighbours again and recompute every face).
constexpr size_t topo_side_cap(size_t n) { return n / 4 + 256; }
constexpr size_t topo_side_bytes(size_t n) { return topo_side_cap(n) * sizeof(TopoSide); }
// FP64 pass: two polygon buffers of 2 x PTM_TOPO_VMAX doubles per thread
constexpr size_t topo64_smem_bytes() { return (size_t)PTM_BLOCK * 4 * PTM_TOPO_VMAX * sizeof(double); }
#define PTM_TOPO64_BLOCKS_PER_SM 4     // 4 x (48 KB + 1 KB) of shared memory

constexpr size_t topo_smem_bytes() { return (size_t)PTM_BLOCK * PTM_TOPO_WORDS * 4; }

}  // namespace ptm
