/*
 * ptm_oracle.c -- plain, slow, FP64 CPU oracle for Polyhedral Template Matching
 * (Larsen, Schmidt & Schiotz, "Robust Structural Identification via Polyhedral
 * Template Matching").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this library.  It shares no code, header or table
 * with the CUDA path: every template, triangulation, rotation group and code it
 * uses is generated here, by brute force, from the definitions in the paper.
 *
 * What it computes, per atom (Algorithm 1, Euclidean neighbour ordering):
 *   1. the k nearest periodic images, ordered by (d^2, atom id, image)   (Sec. 3)
 *   2. for each template S in {SC, FCC, HCP, ICO, BCC} (Table 1, k = 6/12/12/12/14):
 *      the convex hull of the first k neighbours, brute force O(k^4) with exact
 *      integer orientation predicates and Simulation of Simplicity   (Sec. 4)
 *   3. the hull is rejected unless all k points are vertices and the centre is
 *      strictly inside                                        (Algorithm 1)
 *   4. every orientation-preserving isomorphism between the hull graph and any
 *      triangulation of the template hull, found by comparing the Weinberg code
 *      of the hull from EVERY directed start edge with the code of each template
 *      triangulation from one fixed start edge     (Sec. 4, Appendix A; no
 *      canonical forms and no symmetry reduction)
 *   5. the scale-invariant RMSD of every such correspondence, Eq. 3-4, by Horn's
 *      quaternion eigenproblem solved with a Jacobi eigensolver (not QCP)
 *   6. the minimum over templates and correspondences, then orientation (Sec. 7),
 *      strain by least squares + left polar decomposition (Sec. 8, Eq. 6-7) and
 *      the binary alloy label (Sec. 6, Table 3).
 *
 * Readings of the paper that it follows where the paper is silent or ambiguous:
 *   R1  the centre atom belongs to both point sets (N = k + 1), at the origin.
 *   R2  the data set v is scaled by s, the template w by 1/l(w) (Eq. 3-4).
 *   R4  neighbour order by squared distance computed in FP64 (float32 positions
 *       widened exactly) by a fixed sequence of IEEE operations without fused
 *       multiply-add (the "distance contract"), ties by atom id then image
 *       vector: the paper orders by distance and fixes no precision.
 *   R7  hull predicates are exact on integer coordinates quantised at 2^-19 of the
 *       largest component of the FP64 contract vectors (power-of-two grid, round
 *       half to even), with Simulation of Simplicity (priority = neighbour rank)
 *       on exact zeros.
 *   R9  Weinberg walk rules, counter-clockwise rotation seen from outside.
 *   R12 the reported correspondence is the lexicographically smallest member of
 *       its orbit under the template's rotation group.
 *   R13 ties: RMSD^2 within 1e-12 -> earlier template (SC, FCC, HCP, ICO, BCC),
 *       then smaller canonical correspondence.
 *   R15 strain: A^T = pinv(ideal) actual, A = P U, U a proper rotation.
 *   R16 alloy rules of Table 3 for FCC, A2/B2 for BCC (Sec. 6).
 *
 * Compile with -ffp-contract=off: the distance contract forbids fused multiply-add.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NT 5              /* templates: SC, FCC, HCP, ICO, BCC (Algorithm 1 order) */
#define KMAX 14
#define NMAX 15           /* k + 1 points including the centre */
#define CODEMAX 80        /* 2E + 1 <= 73 */
#define QBITS 19          /* quantisation grid: 2^-19 of the largest component */
#define TIE_R2 1e-12

static const int K_OF[NT] = {6, 12, 12, 12, 14};   /* Table 1 */

/* ------------------------------------------------------------------ templates */
/* Raw template shells (Sec. 4, Fig. 2); slot 0 is the centre at the origin. */
static void raw_template(int S, double w[NMAX][3]) {
  memset(w, 0, sizeof(double) * NMAX * 3);
  const double r2 = sqrt(2.0), phi = (1.0 + sqrt(5.0)) / 2.0;
  if (S == 0) {           /* simple cubic: +-x, +-y, +-z */
    static const double t[6][3] = {{1,0,0},{-1,0,0},{0,1,0},{0,-1,0},{0,0,1},{0,0,-1}};
    for (int i = 0; i < 6; i++) for (int c = 0; c < 3; c++) w[1 + i][c] = t[i][c];
  } else if (S == 1) {    /* fcc: (+-1,+-1,0) permutations / sqrt 2 */
    static const double t[12][3] = {{1,1,0},{1,-1,0},{-1,1,0},{-1,-1,0},
                                    {1,0,1},{1,0,-1},{-1,0,1},{-1,0,-1},
                                    {0,1,1},{0,1,-1},{0,-1,1},{0,-1,-1}};
    for (int i = 0; i < 12; i++) for (int c = 0; c < 3; c++) w[1 + i][c] = t[i][c] / r2;
  } else if (S == 2) {    /* hcp: hexagon in z = 0, eclipsed triangles above/below */
    for (int i = 0; i < 6; i++) {
      double a = M_PI / 3.0 * i;
      w[1 + i][0] = cos(a); w[1 + i][1] = sin(a); w[1 + i][2] = 0.0;
    }
    const double rt = 1.0 / sqrt(3.0), h = sqrt(2.0 / 3.0);
    const double ang[3] = {M_PI / 6.0, 5.0 * M_PI / 6.0, 3.0 * M_PI / 2.0};
    for (int i = 0; i < 3; i++) {
      w[7 + i][0] = rt * cos(ang[i]); w[7 + i][1] = rt * sin(ang[i]); w[7 + i][2] = h;
      w[10 + i][0] = rt * cos(ang[i]); w[10 + i][1] = rt * sin(ang[i]); w[10 + i][2] = -h;
    }
  } else if (S == 3) {    /* icosahedron: cyclic permutations of (0, +-1, +-phi) */
    int i = 1;
    for (int s1 = 1; s1 >= -1; s1 -= 2)
      for (int s2 = 1; s2 >= -1; s2 -= 2) {
        double a[3][3] = {{0, s1, s2 * phi}, {s1, s2 * phi, 0}, {s2 * phi, 0, s1}};
        for (int t = 0; t < 3; t++, i++) for (int c = 0; c < 3; c++) w[i][c] = a[t][c];
      }
  } else {                /* bcc: 8 x (+-1/2)^3 then 6 x (+-1,0,0) */
    int i = 1;
    for (int sx = 1; sx >= -1; sx -= 2)
      for (int sy = 1; sy >= -1; sy -= 2)
        for (int sz = 1; sz >= -1; sz -= 2, i++) {
          w[i][0] = 0.5 * sx; w[i][1] = 0.5 * sy; w[i][2] = 0.5 * sz;
        }
    static const double t[6][3] = {{1,0,0},{-1,0,0},{0,1,0},{0,-1,0},{0,0,1},{0,0,-1}};
    for (int j = 0; j < 6; j++) for (int c = 0; c < 3; c++) w[9 + j][c] = t[j][c];
  }
}

/* Translate to the barycentre and scale to mean distance 1 (Eq. 4), N = k + 1. */
static void normalise(int N, const double in[][3], double out[][3]) {
  double b[3] = {0, 0, 0};
  for (int i = 0; i < N; i++) for (int c = 0; c < 3; c++) b[c] += in[i][c];
  for (int c = 0; c < 3; c++) b[c] /= N;
  double l = 0;
  for (int i = 0; i < N; i++) {
    double d[3] = {in[i][0] - b[0], in[i][1] - b[1], in[i][2] - b[2]};
    l += sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  }
  l /= N;
  for (int i = 0; i < N; i++) for (int c = 0; c < 3; c++) out[i][c] = (in[i][c] - b[c]) / l;
}

typedef struct {
  int k;
  double w[NMAX][3];        /* normalised template, slot 0 = centre */
  int ngroup;
  int gperm[60][NMAX];      /* rotation g maps template point s to point gperm[g][s] */
  double gquat[60][4];      /* (w, x, y, z) of rotation g */
  int ntri;
  int (*tri)[3];            /* ntri x (2k-4) facets, vertices = slots 1..k */
  int ncodes;
  uint8_t *codes;           /* ntri codes from the fixed start, CODEMAX bytes each */
  uint8_t *labels;          /* ntri x NMAX: label of slot s (1..k) */
  int *sorted;              /* triangulation indices sorted by code */
  int codelen;
} template_t;

static template_t TPL[NT];
static int initialised = 0;

/* --------------------------------------------------------------- small algebra */
static void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static double det3(const double m[3][3]) {
  return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
       - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
       + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

/* Cyclic Jacobi eigensolver for a symmetric n x n matrix (n <= 4).
   On return a holds the eigenvalues on its diagonal and v the eigenvectors
   in its columns. */
static void jacobi_eigen(int n, double a[4][4], double v[4][4]) {
  for (int i = 0; i < n; i++) for (int j = 0; j < n; j++) v[i][j] = (i == j);
  for (int sweep = 0; sweep < 100; sweep++) {
    double off = 0, diag = 0;
    for (int i = 0; i < n; i++) {
      diag += a[i][i] * a[i][i];
      for (int j = i + 1; j < n; j++) off += a[i][j] * a[i][j];
    }
    if (off <= 1e-34 * (diag + 1e-300)) break;
    for (int p = 0; p < n; p++)
      for (int q = p + 1; q < n; q++) {
        if (a[p][q] == 0.0) continue;
        /* rotation angle that zeroes a[p][q] */
        double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; k++) {          /* columns p, q */
          double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; k++) {          /* rows p, q */
          double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; k++) {
          double vkp = v[k][p], vkq = v[k][q];
          v[k][p] = c * vkp - s * vkq;
          v[k][q] = s * vkp + c * vkq;
        }
      }
  }
}

static void quat_to_matrix(const double q[4], double R[3][3]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

/* Rotation matrix -> unit quaternion: take the largest of the four squared
   components, which is always well conditioned. */
static void matrix_to_quat(const double R[3][3], double q[4]) {
  double t[4] = {1 + R[0][0] + R[1][1] + R[2][2], 1 + R[0][0] - R[1][1] - R[2][2],
                 1 - R[0][0] + R[1][1] - R[2][2], 1 - R[0][0] - R[1][1] + R[2][2]};
  int m = 0;
  for (int i = 1; i < 4; i++) if (t[i] > t[m]) m = i;
  double s = 0.5 / sqrt(t[m]);
  if (m == 0) {
    q[0] = 0.25 / s; q[1] = (R[2][1] - R[1][2]) * s; q[2] = (R[0][2] - R[2][0]) * s; q[3] = (R[1][0] - R[0][1]) * s;
  } else if (m == 1) {
    q[1] = 0.25 / s; q[0] = (R[2][1] - R[1][2]) * s; q[2] = (R[0][1] + R[1][0]) * s; q[3] = (R[0][2] + R[2][0]) * s;
  } else if (m == 2) {
    q[2] = 0.25 / s; q[0] = (R[0][2] - R[2][0]) * s; q[1] = (R[0][1] + R[1][0]) * s; q[3] = (R[1][2] + R[2][1]) * s;
  } else {
    q[3] = 0.25 / s; q[0] = (R[1][0] - R[0][1]) * s; q[1] = (R[0][2] + R[2][0]) * s; q[2] = (R[1][2] + R[2][1]) * s;
  }
  if (q[0] < 0) for (int i = 0; i < 4; i++) q[i] = -q[i];
}

static void quat_mul(const double a[4], const double b[4], double o[4]) {
  o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

/* ---------------------------------------------------------- rotation groups */
/* All proper rotations that map the template shell onto itself, found by trying
   every rotation that sends a fixed independent pair of shell points onto any
   pair with the same lengths and angle. */
static void build_group(template_t *T) {
  const int k = T->k;
  const double tol = 1e-9;
  int a = 1, b = 2;
  { double c[3]; cross3(T->w[a], T->w[b], c);
    while (dot3(c, c) < 1e-6) { b++; cross3(T->w[a], T->w[b], c); } }
  double A[3][3];   /* columns a, b, a x b */
  double ab[3]; cross3(T->w[a], T->w[b], ab);
  for (int c = 0; c < 3; c++) { A[c][0] = T->w[a][c]; A[c][1] = T->w[b][c]; A[c][2] = ab[c]; }
  double dA = det3(A), Ainv[3][3];
  for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) {
    int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
    Ainv[i][j] = (A[i1][j1] * A[i2][j2] - A[i1][j2] * A[i2][j1]) / dA;
  }
  T->ngroup = 0;
  for (int a2 = 1; a2 <= k; a2++)
    for (int b2 = 1; b2 <= k; b2++) {
      if (a2 == b2) continue;
      if (fabs(dot3(T->w[a2], T->w[a2]) - dot3(T->w[a], T->w[a])) > tol) continue;
      if (fabs(dot3(T->w[b2], T->w[b2]) - dot3(T->w[b], T->w[b])) > tol) continue;
      if (fabs(dot3(T->w[a2], T->w[b2]) - dot3(T->w[a], T->w[b])) > tol) continue;
      double B[3][3], ab2[3];
      cross3(T->w[a2], T->w[b2], ab2);
      for (int c = 0; c < 3; c++) { B[c][0] = T->w[a2][c]; B[c][1] = T->w[b2][c]; B[c][2] = ab2[c]; }
      double R[3][3];
      for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) {
        R[i][j] = 0;
        for (int m = 0; m < 3; m++) R[i][j] += B[i][m] * Ainv[m][j];
      }
      if (fabs(det3(R) - 1.0) > 1e-6) continue;
      int perm[NMAX], ok = 1;
      perm[0] = 0;
      for (int s = 1; s <= k && ok; s++) {
        double p[3] = {0, 0, 0};
        for (int i = 0; i < 3; i++) for (int m = 0; m < 3; m++) p[i] += R[i][m] * T->w[s][m];
        int found = -1;
        for (int t = 1; t <= k; t++) {
          double d[3] = {p[0] - T->w[t][0], p[1] - T->w[t][1], p[2] - T->w[t][2]};
          if (dot3(d, d) < 1e-12) { found = t; break; }
        }
        if (found < 0) ok = 0; else perm[s] = found;
      }
      if (!ok) continue;
      int dup = 0;
      for (int g = 0; g < T->ngroup && !dup; g++)
        if (!memcmp(T->gperm[g], perm, sizeof(int) * (k + 1))) dup = 1;
      if (dup) continue;
      memcpy(T->gperm[T->ngroup], perm, sizeof(int) * (k + 1));
      matrix_to_quat(R, T->gquat[T->ngroup]);
      T->ngroup++;
    }
}

/* ------------------------------------------------ exact orientation + SoS */
/* orient(a,b,c,d) = det[b-a; c-a; d-a] on integer coordinates, evaluated exactly
   in 128-bit integers.  Positive means d lies on the side the normal
   (b-a) x (c-a) points to. */
static int sgn128(__int128 x) { return (x > 0) - (x < 0); }

static __int128 orient_exact_val(const int64_t a[3], const int64_t b[3], const int64_t c[3],
                                 const int64_t d[3]) {
  __int128 u[3], v[3], w[3];
  for (int i = 0; i < 3; i++) { u[i] = b[i] - a[i]; v[i] = c[i] - a[i]; w[i] = d[i] - a[i]; }
  return u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0])
       + u[2] * (v[0] * w[1] - v[1] * w[0]);
}

/* Determinant of the square submatrix of M (4 x 4, rows = points (x, y, z, 1))
   keeping rows `rows` and columns `cols` (both of length m), by cofactor expansion. */
static __int128 minor_det(const __int128 M[4][4], const int *rows, const int *cols, int m) {
  if (m == 0) return 1;
  if (m == 1) return M[rows[0]][cols[0]];
  __int128 acc = 0;
  for (int j = 0; j < m; j++) {
    int sr[4], sc[4], t = 0;
    for (int i = 1; i < m; i++) sr[i - 1] = rows[i];
    for (int i = 0; i < m; i++) if (i != j) sc[t++] = cols[i];
    __int128 sub = minor_det(M, sr, sc, m - 1);
    acc += ((j & 1) ? -1 : 1) * M[rows[0]][cols[j]] * sub;
  }
  return acc;
}

/* Simulation of Simplicity (Edelsbrunner & Muecke 1990) for the 4 x 4 matrix
   D = det[[p_r, 1]]_{r=0..3}.  Coordinate c of the point with priority r
   (neighbour rank, 1-based) is perturbed by eps^(2^(3(r-1)+c)).  det(D + E) is
   expanded over all partial matchings S between rows and the perturbed columns
   (generalised Laplace expansion); each matching gives a monomial with a unique
   exponent (the bit mask) and the coefficient (-1)^(sum rows + sum cols) sgn(sigma)
   det(D without the rows and columns of S).  The sign of the perturbed
   determinant is the sign of the nonzero coefficient with the smallest mask. */
static int sos_det4_sign(const int64_t p[4][3], const int prio[4]) {
  __int128 M[4][4];
  for (int r = 0; r < 4; r++) { for (int c = 0; c < 3; c++) M[r][c] = p[r][c]; M[r][3] = 1; }
  uint64_t best_mask = UINT64_MAX;
  int best_sign = 0;
  int asg[4];
  for (int code = 0; code < 256; code++) {
    int used[3] = {0, 0, 0}, ok = 1;
    for (int r = 0; r < 4; r++) {
      asg[r] = ((code >> (2 * r)) & 3) - 1;          /* -1 = row not in S */
      if (asg[r] >= 0) { if (used[asg[r]]) ok = 0; used[asg[r]] = 1; }
    }
    if (!ok) continue;
    uint64_t mask = 0;
    int C[4], m = 0, keepr[4], keepc[4], nk = 0, nkc = 0, srow = 0, scol = 0;
    for (int r = 0; r < 4; r++) {
      if (asg[r] >= 0) {
        mask |= 1ULL << (3 * (prio[r] - 1) + asg[r]);
        C[m] = asg[r]; m++;
        srow += r; scol += asg[r];
      } else keepr[nk++] = r;
    }
    for (int c = 0; c < 4; c++) {
      int inS = 0;
      for (int i = 0; i < m; i++) if (C[i] == c) inS = 1;
      if (!inS) keepc[nkc++] = c;
    }
    if (mask >= best_mask) continue;
    __int128 mdet = minor_det(M, keepr, keepc, nk);
    if (mdet == 0) continue;
    int inv = 0;                                     /* sign of sigma: rows R sorted ascending */
    for (int i = 0; i < m; i++) for (int j = i + 1; j < m; j++) if (C[i] > C[j]) inv++;
    int s = (((srow + scol) & 1) ? -1 : 1) * ((inv & 1) ? -1 : 1) * sgn128(mdet);
    best_mask = mask;
    best_sign = s;
  }
  return best_sign;
}

/* Orientation of four quantised points with SoS; never zero. */
static int orient_sos(const int64_t a[3], const int64_t b[3], const int64_t c[3],
                      const int64_t d[3], const int prio[4]) {
  int s = sgn128(orient_exact_val(a, b, c, d));
  if (s) return s;
  int64_t p[4][3];
  memcpy(p[0], a, 24); memcpy(p[1], b, 24); memcpy(p[2], c, 24); memcpy(p[3], d, 24);
  return -sos_det4_sign(p, prio);                   /* orient = -det[[p, 1]] */
}

int ptmo_orient(const int64_t *a, const int64_t *b, const int64_t *c, const int64_t *d,
                const int *prio) {
  return orient_sos(a, b, c, d, prio);
}
int ptmo_orient_exact(const int64_t *a, const int64_t *b, const int64_t *c, const int64_t *d) {
  return sgn128(orient_exact_val(a, b, c, d));
}

/* --------------------------------------------------------- brute-force hull */
/* Triangulated convex hull of k quantised points with SoS (priority = index + 1):
   a triple is a facet iff every other point lies strictly on one side.  Facets
   are emitted counter-clockwise seen from outside.  Returns the number of facets,
   or -1 if some point is not a hull vertex. */
int ptmo_hull(const int64_t *q, int k, int *facets) {
  int nf = 0, isv[KMAX] = {0};
  for (int i = 0; i < k; i++)
    for (int j = i + 1; j < k; j++)
      for (int l = j + 1; l < k; l++) {
        int pos = 0, neg = 0;
        for (int m = 0; m < k; m++) {
          if (m == i || m == j || m == l) continue;
          int prio[4] = {i + 1, j + 1, l + 1, m + 1};
          int s = orient_sos(q + 3 * i, q + 3 * j, q + 3 * l, q + 3 * m, prio);
          if (s > 0) pos++; else neg++;
        }
        if (pos && neg) continue;
        if (nf == 32) return -2;
        if (pos == 0) { facets[3 * nf] = i; facets[3 * nf + 1] = j; facets[3 * nf + 2] = l; }
        else          { facets[3 * nf] = i; facets[3 * nf + 1] = l; facets[3 * nf + 2] = j; }
        nf++;
        isv[i] = isv[j] = isv[l] = 1;
      }
  for (int i = 0; i < k; i++) if (!isv[i]) return -1;
  return nf;
}

/* -------------------------------------------------------------- Weinberg codes */
/* third[u][v] = w when (u, v, w) is a facet (counter-clockwise from outside).
   Around vertex v the counter-clockwise successor of neighbour u is third[v][u]. */
static void build_third(int nv, int nf, const int *facets, int third[KMAX][KMAX]) {
  for (int i = 0; i < nv; i++) for (int j = 0; j < nv; j++) third[i][j] = -1;
  for (int f = 0; f < nf; f++) {
    int a = facets[3 * f], b = facets[3 * f + 1], c = facets[3 * f + 2];
    third[a][b] = c; third[b][c] = a; third[c][a] = b;
  }
}

/* Weinberg's walk from the directed start edge u -> v.  Rules:
     arriving at a new vertex: leave by the next edge counter-clockwise after the
       arrival edge;
     arriving at an old vertex along an edge not yet walked in either direction:
       walk back along it;
     otherwise: leave by the first unused edge counter-clockwise after the arrival
       edge.
   Vertices are labelled 1, 2, ... in order of first visit; the code is the label
   sequence.  Returns the code length (2E + 1 when the walk covers every edge in
   both directions).  label_out[v] receives the label of vertex v. */
static int weinberg(int nv, int third[KMAX][KMAX], int u, int v, uint8_t *code,
                    uint8_t *label_out) {
  uint8_t label[KMAX] = {0};
  uint8_t used[KMAX][KMAX];
  memset(used, 0, sizeof used);
  int next = 1, len = 0;
  label[u] = next++;
  code[len++] = label[u];
  used[u][v] = 1;
  int isnew = !label[v];
  if (isnew) label[v] = next++;
  code[len++] = label[v];
  for (;;) {
    int w = -1;
    if (isnew) {
      w = third[v][u];
    } else if (!used[v][u]) {
      w = u;
    } else {
      int x = third[v][u];
      while (x != u && x >= 0) {
        if (!used[v][x]) { w = x; break; }
        x = third[v][x];
      }
    }
    if (w < 0) break;
    used[v][w] = 1;
    u = v; v = w;
    isnew = !label[v];
    if (isnew) label[v] = next++;
    code[len++] = label[v];
    if (len >= CODEMAX) break;
  }
  if (label_out) memcpy(label_out, label, nv);
  return len;
}

int ptmo_weinberg(int nv, int nf, const int *facets, int u, int v, uint8_t *code, uint8_t *label) {
  int third[KMAX][KMAX];
  build_third(nv, nf, facets, third);
  if (third[u][v] < 0) return -1;
  return weinberg(nv, third, u, v, code, label);
}

/* -------------------------------------------------- template triangulations */
/* Faces of the template hull found geometrically: every plane through three
   shell points with all others on or behind it; coplanar points join the face.
   Each 4-gon face (fcc/hcp squares, bcc rhombi) has two triangulations (Sec. 4). */
static int build_triangulations(template_t *T) {
  const int k = T->k;
  const double tol = 1e-9;
  uint32_t facemask[64];
  double facenorm[64][3];
  int nface = 0;
  for (int i = 1; i <= k; i++)
    for (int j = i + 1; j <= k; j++)
      for (int l = j + 1; l <= k; l++) {
        double u[3], v[3], n[3];
        for (int c = 0; c < 3; c++) { u[c] = T->w[j][c] - T->w[i][c]; v[c] = T->w[l][c] - T->w[i][c]; }
        cross3(u, v, n);
        double nn = sqrt(dot3(n, n));
        if (nn < 1e-9) continue;
        for (int c = 0; c < 3; c++) n[c] /= nn;
        int pos = 0, neg = 0;
        uint32_t mask = (1u << i) | (1u << j) | (1u << l);
        for (int m = 1; m <= k; m++) {
          if (m == i || m == j || m == l) continue;
          double d[3] = {T->w[m][0] - T->w[i][0], T->w[m][1] - T->w[i][1], T->w[m][2] - T->w[i][2]};
          double s = dot3(n, d);
          if (s > tol) pos++; else if (s < -tol) neg++; else mask |= 1u << m;
        }
        if (pos && neg) continue;
        if (pos) for (int c = 0; c < 3; c++) n[c] = -n[c];   /* outward normal */
        int dup = 0;
        for (int f = 0; f < nface; f++) if (facemask[f] == mask) dup = 1;
        if (dup) continue;
        facemask[nface] = mask;
        memcpy(facenorm[nface], n, sizeof n);
        nface++;
      }
  /* order each face's vertices counter-clockwise about its outward normal */
  int fv[64][4], fn[64], quads[16], nquad = 0;
  for (int f = 0; f < nface; f++) {
    int idx[8], m = 0;
    for (int s = 1; s <= k; s++) if (facemask[f] >> s & 1) idx[m++] = s;
    if (m > 4) return -1;
    double cen[3] = {0, 0, 0};
    for (int t = 0; t < m; t++) for (int c = 0; c < 3; c++) cen[c] += T->w[idx[t]][c] / m;
    double e1[3], e2[3];
    for (int c = 0; c < 3; c++) e1[c] = T->w[idx[0]][c] - cen[c];
    cross3(facenorm[f], e1, e2);
    double ang[8];
    for (int t = 0; t < m; t++) {
      double d[3] = {T->w[idx[t]][0] - cen[0], T->w[idx[t]][1] - cen[1], T->w[idx[t]][2] - cen[2]};
      ang[t] = atan2(dot3(d, e2), dot3(d, e1));
    }
    for (int a = 0; a < m; a++) for (int b = a + 1; b < m; b++)
      if (ang[b] < ang[a]) { double ta = ang[a]; ang[a] = ang[b]; ang[b] = ta;
                             int ti = idx[a]; idx[a] = idx[b]; idx[b] = ti; }
    for (int t = 0; t < m; t++) fv[f][t] = idx[t];
    fn[f] = m;
    if (m == 4) quads[nquad++] = f;
  }
  T->ntri = 1 << nquad;
  const int nfac = 2 * k - 4;
  T->tri = malloc(sizeof(int[3]) * (size_t)T->ntri * nfac);
  for (int t = 0; t < T->ntri; t++) {
    int (*out)[3] = T->tri + (size_t)t * nfac, o = 0;
    for (int f = 0; f < nface; f++) {
      if (fn[f] == 3) { out[o][0] = fv[f][0]; out[o][1] = fv[f][1]; out[o][2] = fv[f][2]; o++; continue; }
      int qi = 0;
      while (quads[qi] != f) qi++;
      int *p = fv[f];
      if ((t >> qi & 1) == 0) {
        out[o][0] = p[0]; out[o][1] = p[1]; out[o][2] = p[2]; o++;
        out[o][0] = p[0]; out[o][1] = p[2]; out[o][2] = p[3]; o++;
      } else {
        out[o][0] = p[1]; out[o][1] = p[2]; out[o][2] = p[3]; o++;
        out[o][0] = p[1]; out[o][1] = p[3]; out[o][2] = p[0]; o++;
      }
    }
    if (o != nfac) return -2;
  }
  return 0;
}

static const template_t *cmp_tpl;
static int cmp_codes(const void *a, const void *b) {
  int ia = *(const int *)a, ib = *(const int *)b;
  int c = memcmp(cmp_tpl->codes + (size_t)ia * CODEMAX, cmp_tpl->codes + (size_t)ib * CODEMAX,
                 cmp_tpl->codelen);
  return c ? c : (ia - ib);
}

/* Weinberg code of every template triangulation from one fixed start edge
   (slot 1 to its lowest-numbered neighbour); codes are sorted for lookup. */
static int build_codes(template_t *T) {
  const int k = T->k, nfac = 2 * k - 4;
  T->codes = calloc((size_t)T->ntri, CODEMAX);
  T->labels = calloc((size_t)T->ntri, NMAX);
  T->sorted = malloc(sizeof(int) * T->ntri);
  for (int t = 0; t < T->ntri; t++) {
    int f0[3 * 24];
    for (int f = 0; f < nfac; f++) for (int c = 0; c < 3; c++) f0[3 * f + c] = T->tri[(size_t)t * nfac + f][c] - 1;
    int third[KMAX][KMAX];
    build_third(k, nfac, f0, third);
    int v0 = -1;
    for (int v = 0; v < k && v0 < 0; v++) if (third[0][v] >= 0) v0 = v;
    uint8_t lab[KMAX];
    int len = weinberg(k, third, 0, v0, T->codes + (size_t)t * CODEMAX, lab);
    if (len != 2 * (3 * k - 6) + 1) return -3;
    T->codelen = len;
    for (int s = 0; s < k; s++) T->labels[(size_t)t * NMAX + 1 + s] = lab[s];
    T->sorted[t] = t;
  }
  cmp_tpl = T;
  qsort(T->sorted, T->ntri, sizeof(int), cmp_codes);
  return 0;
}

int ptmo_init(void) {
  if (initialised) return 0;
  for (int S = 0; S < NT; S++) {
    template_t *T = &TPL[S];
    T->k = K_OF[S];
    double raw[NMAX][3];
    raw_template(S, raw);
    normalise(T->k + 1, raw, T->w);
    build_group(T);
    int rc = build_triangulations(T);
    if (rc) return 10 * S + rc;
    rc = build_codes(T);
    if (rc) return 10 * S + rc;
  }
  initialised = 1;
  return 0;
}

/* ------------------------------------------------- accessors for the tests */
int ptmo_template(int S, double *w, int *k) {
  if (ptmo_init()) return -1;
  *k = TPL[S].k;
  memcpy(w, TPL[S].w, sizeof(double) * 3 * (TPL[S].k + 1));
  return 0;
}
int ptmo_group(int S, int *perms, double *quats) {
  if (ptmo_init()) return -1;
  const template_t *T = &TPL[S];
  for (int g = 0; g < T->ngroup; g++) {
    for (int s = 0; s <= T->k; s++) perms[g * (T->k + 1) + s] = T->gperm[g][s];
    for (int c = 0; c < 4; c++) quats[4 * g + c] = T->gquat[g][c];
  }
  return T->ngroup;
}
int ptmo_n_triangulations(int S) { return ptmo_init() ? -1 : TPL[S].ntri; }
int ptmo_triangulation(int S, int t, int *facets) {
  if (ptmo_init()) return -1;
  const template_t *T = &TPL[S];
  const int nfac = 2 * T->k - 4;
  for (int f = 0; f < nfac; f++) for (int c = 0; c < 3; c++) facets[3 * f + c] = T->tri[(size_t)t * nfac + f][c];
  return nfac;
}

/* -------------------------------------------------------------- superposition */
/* Eq. 3 for paired points: data v (N x 3, rows paired with template rows w,
   w already normalised by Eq. 4).  The data are translated to their barycentre;
   the rotation Q of the template and the scale s of the data minimise
   sum |s v'_i - Q w_i|^2.  Q maximises sum v'_i . Q w_i, the largest eigenvalue
   of Horn's symmetric 4 x 4 matrix; s = lambda / sum |v'|^2 (Horn 1987).
   Returns RMSD^2 evaluated explicitly at the optimum. */
double ptmo_superpose(int N, const double *v, const double *w, double *quat, double *scale,
                      double *lambda_out) {
  double vb[3] = {0, 0, 0}, wb[3] = {0, 0, 0};
  for (int i = 0; i < N; i++) for (int c = 0; c < 3; c++) { vb[c] += v[3 * i + c] / N; wb[c] += w[3 * i + c] / N; }
  double S[3][3] = {{0}}, Gv = 0;
  for (int i = 0; i < N; i++) {
    double vp[3], wp[3];
    for (int c = 0; c < 3; c++) { vp[c] = v[3 * i + c] - vb[c]; wp[c] = w[3 * i + c] - wb[c]; }
    Gv += dot3(vp, vp);
    for (int a = 0; a < 3; a++) for (int b = 0; b < 3; b++) S[a][b] += wp[a] * vp[b];
  }
  double K[4][4] = {
    {S[0][0] + S[1][1] + S[2][2], S[1][2] - S[2][1], S[2][0] - S[0][2], S[0][1] - S[1][0]},
    {S[1][2] - S[2][1], S[0][0] - S[1][1] - S[2][2], S[0][1] + S[1][0], S[2][0] + S[0][2]},
    {S[2][0] - S[0][2], S[0][1] + S[1][0], -S[0][0] + S[1][1] - S[2][2], S[1][2] + S[2][1]},
    {S[0][1] - S[1][0], S[2][0] + S[0][2], S[1][2] + S[2][1], -S[0][0] - S[1][1] + S[2][2]}};
  double V[4][4];
  jacobi_eigen(4, K, V);
  int m = 0;
  for (int i = 1; i < 4; i++) if (K[i][i] > K[m][m]) m = i;
  double lam = K[m][m];
  double q[4] = {V[0][m], V[1][m], V[2][m], V[3][m]};
  double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int i = 0; i < 4; i++) q[i] /= nq;
  if (q[0] < 0) for (int i = 0; i < 4; i++) q[i] = -q[i];
  double s = Gv > 0 ? lam / Gv : 0.0;
  double R[3][3];
  quat_to_matrix(q, R);
  double r2 = 0;
  for (int i = 0; i < N; i++) {
    double vp[3], wp[3], Rw[3];
    for (int c = 0; c < 3; c++) { vp[c] = v[3 * i + c] - vb[c]; wp[c] = w[3 * i + c] - wb[c]; }
    for (int a = 0; a < 3; a++) Rw[a] = R[a][0] * wp[0] + R[a][1] * wp[1] + R[a][2] * wp[2];
    for (int c = 0; c < 3; c++) { double d = s * vp[c] - Rw[c]; r2 += d * d; }
  }
  if (quat) memcpy(quat, q, sizeof q);
  if (scale) *scale = s;
  if (lambda_out) *lambda_out = lam;
  return r2 / N;
}

/* ------------------------------------------------------------------- strain */
/* Left polar decomposition A = P U (Sec. 8): P = X diag(sigma) X^T from the
   eigen-decomposition A A^T = X diag(sigma^2) X^T; when det A < 0 the smallest
   singular value changes sign so that U = P^-1 A is a proper rotation. */
void ptmo_polar(const double *A, double *P, double *U) {
  double AA[4][4] = {{0}}, X[4][4];
  for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) {
    double s = 0;
    for (int m = 0; m < 3; m++) s += A[3 * i + m] * A[3 * j + m];
    AA[i][j] = s;
  }
  jacobi_eigen(3, AA, X);
  double sig[3];
  int imin = 0;
  for (int i = 0; i < 3; i++) { sig[i] = sqrt(AA[i][i] > 0 ? AA[i][i] : 0); if (sig[i] < sig[imin]) imin = i; }
  double Am[3][3];
  for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) Am[i][j] = A[3 * i + j];
  if (det3(Am) < 0) sig[imin] = -sig[imin];
  for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) {
    double s = 0;
    for (int m = 0; m < 3; m++) s += X[i][m] * sig[m] * X[j][m];
    P[3 * i + j] = s;
  }
  if (U) {   /* U = P^-1 A via the same eigenvectors */
    for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) {
      double s = 0;
      for (int m = 0; m < 3; m++) {
        double xa = 0;
        for (int t = 0; t < 3; t++) xa += X[t][m] * A[3 * t + j];
        s += X[i][m] * (sig[m] != 0 ? xa / sig[m] : 0.0);
      }
      U[3 * i + j] = s;
    }
  }
}

/* ------------------------------------------------------ neighbours (Sec. 3) */
typedef struct { double d2; int32_t j; int32_t n[3]; double dr[3]; } cand_t;   /* dr: contract vector */

static int cmp_cand(const void *a, const void *b) {
  const cand_t *x = a, *y = b;
  if (x->d2 != y->d2) return x->d2 < y->d2 ? -1 : 1;
  if (x->j != y->j) return x->j < y->j ? -1 : 1;
  for (int c = 0; c < 3; c++) if (x->n[c] != y->n[c]) return x->n[c] < y->n[c] ? -1 : 1;
  return 0;
}

typedef struct {
  const void *pos; int f64; int64_t n;
  double H[9], Hinv[9], width[3];
  uint8_t pbc[3];
  double *frac;             /* n x 3 fractional coordinates (image search only) */
} frame_t;

/* Shift of image n: (n0 H0 + n1 H1) + n2 H2 per component, FP64, no FMA. */
static void shift64(const double *H, const int32_t n[3], double s[3]) {
  for (int c = 0; c < 3; c++) s[c] = ((double)n[0] * H[c] + (double)n[1] * H[3 + c]) + (double)n[2] * H[6 + c];
}

/* The distance contract: neighbour vector and squared length in FP64, one IEEE
   operation at a time, in this order (float32 positions are first widened to
   double, which is exact):
     dr_c = (x_j,c - x_i,c) + shift_c
     d2   = (dr_x dr_x + dr_y dr_y) + dr_z dr_z
   The paper orders neighbours by distance (Sec. 3, Table 1) and fixes no
   precision; the plain definition is the distance between the given points, so
   the order is decided in FP64 whatever the input type.                        */
static double posval(const frame_t *F, int64_t i, int c);
static double contract(const frame_t *F, int64_t i, int64_t j, const int32_t n[3], double drc[3]) {
  double s[3];
  shift64(F->H, n, s);
  double d[3];
  for (int c = 0; c < 3; c++) {
    double t = posval(F, j, c) - posval(F, i, c);
    d[c] = t + s[c];
    drc[c] = d[c];
  }
  double a = d[0] * d[0], b = d[1] * d[1], e = d[2] * d[2];
  double ab = a + b;
  return ab + e;
}

static double posval(const frame_t *F, int64_t i, int c) {
  return F->f64 ? ((const double *)F->pos)[3 * i + c] : (double)((const float *)F->pos)[3 * i + c];
}

static void frame_setup(frame_t *F) {
  const double *H = F->H;
  double det = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6])
             + H[2] * (H[3] * H[7] - H[4] * H[6]);
  for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) {
    int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
    F->Hinv[3 * i + j] = (H[3 * i1 + j1] * H[3 * i2 + j2] - H[3 * i1 + j2] * H[3 * i2 + j1]) / det;
  }
  for (int c = 0; c < 3; c++) {
    double g = 0;
    for (int r = 0; r < 3; r++) g += F->Hinv[3 * r + c] * F->Hinv[3 * r + c];
    F->width[c] = 1.0 / sqrt(g);
  }
  F->frac = malloc(sizeof(double) * 3 * (size_t)F->n);
  for (int64_t i = 0; i < F->n; i++)
    for (int c = 0; c < 3; c++) {
      double f = 0;
      for (int r = 0; r < 3; r++) f += posval(F, i, r) * F->Hinv[3 * r + c];
      F->frac[3 * i + c] = f;
    }
}

/* Brute force over every atom and every image within a cutoff radius R; the
   cutoff doubles until the kmax-th neighbour lies safely inside it. */
static int knn(const frame_t *F, int64_t i, int kmax, cand_t *out) {
  double vol = fabs(F->H[0] * (F->H[4] * F->H[8] - F->H[5] * F->H[7])
                  - F->H[1] * (F->H[3] * F->H[8] - F->H[5] * F->H[6])
                  + F->H[2] * (F->H[3] * F->H[7] - F->H[4] * F->H[6]));
  double rho = F->n / vol;
  double R = cbrt(3.0 * (kmax + 8) / (4.0 * M_PI * rho));
  size_t cap = 256;
  cand_t *c = malloc(sizeof(cand_t) * cap);
  for (int attempt = 0; attempt < 40; attempt++, R *= 1.5) {
    size_t nc = 0;
    double R2 = R * R;
    for (int64_t j = 0; j < F->n; j++) {
      int lo[3], hi[3];
      for (int d = 0; d < 3; d++) {
        if (!F->pbc[d]) { lo[d] = hi[d] = 0; continue; }
        double df = F->frac[3 * j + d] - F->frac[3 * i + d];
        double rr = R / F->width[d] * (1 + 1e-9) + 1e-12;
        lo[d] = (int)ceil(-df - rr);
        hi[d] = (int)floor(-df + rr);
      }
      int32_t n[3];
      for (n[0] = lo[0]; n[0] <= hi[0]; n[0]++)
        for (n[1] = lo[1]; n[1] <= hi[1]; n[1]++)
          for (n[2] = lo[2]; n[2] <= hi[2]; n[2]++) {
            if (j == i && !n[0] && !n[1] && !n[2]) continue;
            double drc[3];
            double d2 = contract(F, i, j, n, drc);
            if (d2 > R2) continue;
            if (nc == cap) { cap *= 2; c = realloc(c, sizeof(cand_t) * cap); }
            cand_t *e = &c[nc++];
            e->d2 = d2; e->j = (int32_t)j; memcpy(e->n, n, sizeof n); memcpy(e->dr, drc, sizeof drc);
          }
    }
    qsort(c, nc, sizeof(cand_t), cmp_cand);
    /* complete when the kmax-th contract distance is safely inside the cutoff,
       or when every atom of a non-periodic system has been seen */
    int all_np = !F->pbc[0] && !F->pbc[1] && !F->pbc[2];
    if ((int64_t)nc >= kmax && c[kmax - 1].d2 < R2 * (1 - 1e-3)) {
      memcpy(out, c, sizeof(cand_t) * kmax);
      free(c);
      return kmax;
    }
    if (all_np && (int64_t)nc >= F->n - 1 && R > 1e3 * cbrt(vol)) {
      int m = (int)(nc < (size_t)kmax ? nc : (size_t)kmax);
      memcpy(out, c, sizeof(cand_t) * m);
      free(c);
      return m;
    }
  }
  free(c);
  return -1;
}

/* ---------------------------------------- topological ordering (Sec. 3, Eq. 5) */
#define TOPO_N 18          /* neighbours whose Voronoi faces are measured (Sec. 9) */
#define TOPO_BAND 1e-3     /* areas closer than this x the mean squared distance tie */

/* Area of the face between the Voronoi cell of the origin and that of point j,
   the cell taken among the m points v (the origin's neighbours): the bisector
   plane x.v_j = |v_j|^2 / 2, clipped by every other half-space
   x.v_i <= |v_i|^2 / 2.  The plane is parametrised by an orthonormal basis,
   a square of half-width R (far outside any bounded cell) is clipped one
   half-plane at a time, and the area is the shoelace formula; 0 when nothing
   is left (the cells are not adjacent). */
static double voronoi_face_area(int m, const double (*v)[3], int j, double R) {
  double n[3] = {v[j][0], v[j][1], v[j][2]};
  double nn = sqrt(dot3(n, n));
  double u[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
  double a[3] = {fabs(u[0]) < 0.6 ? 1.0 : 0.0, fabs(u[0]) < 0.6 ? 0.0 : 1.0, 0.0};
  double e1[3], e2[3];
  cross3(u, a, e1);
  double l1 = sqrt(dot3(e1, e1));
  for (int c = 0; c < 3; c++) e1[c] /= l1;
  cross3(u, e1, e2);
  double p0[3] = {0.5 * n[0], 0.5 * n[1], 0.5 * n[2]};
  double P[64][2], Q[64][2];
  int np = 4;
  P[0][0] = -R; P[0][1] = -R; P[1][0] = R; P[1][1] = -R; P[2][0] = R; P[2][1] = R; P[3][0] = -R; P[3][1] = R;
  for (int i = 0; i < m && np > 0; i++) {
    if (i == j) continue;
    /* v_i . (p0 + s e1 + t e2) <= |v_i|^2 / 2   <=>   A s + B t <= Cc */
    double A = dot3(v[i], e1), B = dot3(v[i], e2), Cc = 0.5 * dot3(v[i], v[i]) - dot3(v[i], p0);
    int nq = 0;
    for (int k = 0; k < np; k++) {
      const double *x = P[k], *y = P[(k + 1) % np];
      double fx = A * x[0] + B * x[1] - Cc, fy = A * y[0] + B * y[1] - Cc;
      if (fx <= 0 && nq < 64) { Q[nq][0] = x[0]; Q[nq][1] = x[1]; nq++; }
      if (((fx < 0 && fy > 0) || (fx > 0 && fy < 0)) && nq < 64) {
        double t = fx / (fx - fy);
        Q[nq][0] = x[0] + t * (y[0] - x[0]); Q[nq][1] = x[1] + t * (y[1] - x[1]); nq++;
      }
    }
    np = nq;
    memcpy(P, Q, sizeof(double) * 2 * nq);
  }
  double s2 = 0;
  for (int k = 0; k < np; k++) s2 += P[k][0] * P[(k + 1) % np][1] - P[(k + 1) % np][0] * P[k][1];
  return fabs(0.5 * s2);
}

typedef struct { double area; int rank; } topo_t;
static int cmp_topo(const void *a, const void *b) {
  const topo_t *x = a, *y = b;
  if (x->area != y->area) return x->area > y->area ? -1 : 1;
  return x->rank - y->rank;
}

/* Reorder the m Euclidean-ordered neighbours nb (m <= TOPO_N) by Eq. 5: face
   area of the Voronoi cell descending, then distance.  Areas are grouped when
   consecutive ones (in descending order) differ by at most TOPO_BAND x the
   mean squared neighbour distance; inside a group the Euclidean order (distance,
   then atom id, then image) decides.  FP64 exact neighbour vectors. */
static void topo_order(int m, cand_t *nb, double *areas_out) {
  double v[TOPO_N][3], mean2 = 0, dmax = 0;
  for (int t = 0; t < m; t++) {
    for (int c = 0; c < 3; c++) v[t][c] = nb[t].dr[c];
    double d2 = dot3(v[t], v[t]);
    mean2 += d2;
    if (d2 > dmax) dmax = d2;
  }
  mean2 /= m;
  double R = 10.0 * sqrt(dmax);
  topo_t T[TOPO_N];
  for (int t = 0; t < m; t++) { T[t].area = voronoi_face_area(m, (const double (*)[3])v, t, R); T[t].rank = t; }
  if (areas_out) for (int t = 0; t < m; t++) areas_out[t] = T[t].area;
  qsort(T, m, sizeof(topo_t), cmp_topo);
  /* group ids by the band, then order by (group, Euclidean rank) */
  int group[TOPO_N];
  for (int t = 0, g = 0; t < m; t++) {
    if (t > 0 && T[t - 1].area - T[t].area > TOPO_BAND * mean2) g++;
    group[T[t].rank] = g;
  }
  int order[TOPO_N], k = 0;
  for (int g = 0; k < m; g++)
    for (int t = 0; t < m; t++) if (group[t] == g) order[k++] = t;
  cand_t tmp[TOPO_N];
  for (int t = 0; t < m; t++) tmp[t] = nb[order[t]];
  memcpy(nb, tmp, sizeof(cand_t) * m);
}

/* A frame handle holds the positions (not copied), the cell and the fractional
   coordinates used to bound the image search; it is read-only afterwards, so
   several threads may classify disjoint atom lists of one frame at once. */
void *ptmo_frame_new(const void *pos, int f64, int64_t n, const double *cell, const uint8_t *pbc) {
  frame_t *F = calloc(1, sizeof(frame_t));
  F->pos = pos; F->f64 = f64; F->n = n;
  memcpy(F->H, cell, sizeof F->H);
  for (int c = 0; c < 3; c++) F->pbc[c] = pbc[c];
  frame_setup(F);
  return F;
}

void ptmo_frame_free(void *h) {
  frame_t *F = h;
  if (!F) return;
  free(F->frac);
  free(F);
}

int ptmo_knn(void *h, int64_t atom, int kmax, int32_t *ids, int32_t *imgs, double *dr, double *d2) {
  const frame_t *F = h;
  cand_t c[64];
  if (kmax > 64) return -1;
  int m = knn(F, atom, kmax, c);
  for (int t = 0; t < m; t++) {
    ids[t] = c[t].j;
    for (int d = 0; d < 3; d++) { imgs[3 * t + d] = c[t].n[d]; dr[3 * t + d] = c[t].dr[d]; }
    d2[t] = c[t].d2;
  }
  return m;
}

/* Quantisation for the exact hull predicates: q = rint(dr * 2^(19 - e)) with 2^e > max |dr component| over
   the given neighbours.  The scaling is exact; rint rounds half to even. */
int ptmo_quantise(int m, const double *drc, int64_t *q) {
  double mx = 0;
  for (int t = 0; t < 3 * m; t++) if (fabs(drc[t]) > mx) mx = fabs(drc[t]);
  int e = 0;
  frexp(mx, &e);
  double sc = ldexp(1.0, QBITS - e);
  for (int t = 0; t < 3 * m; t++) q[t] = llrint(drc[t] * sc);
  return e;
}

/* --------------------------------------------------------- classification */
typedef struct {
  double r2; int S; uint8_t cp[NMAX];   /* canonical correspondence: neighbour rank per slot */
  double quat[4]; double scale; int perm[NMAX];   /* perm[j] = slot of neighbour rank j */
} candidate_t;

/* Lexicographically smallest member of the orbit {s -> corr[g(s)] : g in G}. */
static void canonical_corr(const template_t *T, const int *corr, uint8_t *best) {
  int k = T->k;
  uint8_t cur[NMAX];
  for (int g = 0; g < T->ngroup; g++) {
    for (int s = 0; s <= k; s++) cur[s] = (uint8_t)corr[T->gperm[g][s]];
    if (g == 0 || memcmp(cur, best, k + 1) < 0) memcpy(best, cur, k + 1);
  }
}

static int better(const candidate_t *a, const candidate_t *b, int k_of_b) {
  (void)k_of_b;
  if (a->S != b->S) return a->S < b->S;
  return memcmp(a->cp, b->cp, K_OF[a->S] + 1) < 0;
}

typedef struct {
  int8_t structure, alloy;
  double rmsd, scale, quat[4], strain[9];
  int32_t corr[NMAX];
  int ncand;
  int32_t nbr[KMAX];
} result_t;

static void alloy_label(int S, const uint8_t *cp, const int32_t *nid, int64_t centre,
                        const int8_t *species, int8_t *out) {
  *out = 0;
  if (!species) return;
  int8_t c = species[centre];
  if (S == 1) {
    /* Table 3: template slots 1-4 lie in z = 0, 5-8 in y = 0, 9-12 in x = 0 */
    int same_planes = 0, other_planes = 0;
    for (int p = 0; p < 3; p++) {
      int same = 0;
      for (int s = 1 + 4 * p; s <= 4 + 4 * p; s++) same += species[nid[cp[s] - 1]] == c;
      if (same == 4) same_planes++;
      else if (same == 0) other_planes++;
    }
    if (same_planes == 3) *out = 1;                              /* A1 */
    else if (same_planes == 1 && other_planes == 2) *out = 2;    /* L1_0 */
    else if (same_planes == 2 && other_planes == 1) *out = 3;    /* L1_2, majority site */
    else if (other_planes == 3) *out = 4;                        /* L1_2, minority site */
  } else if (S == 4) {
    int inner_same = 0, outer_same = 0;
    for (int s = 1; s <= 8; s++) inner_same += species[nid[cp[s] - 1]] == c;
    for (int s = 9; s <= 14; s++) outer_same += species[nid[cp[s] - 1]] == c;
    if (inner_same == 8 && outer_same == 6) *out = 1;            /* A2 */
    else if (inner_same == 0 && outer_same == 6) *out = 5;       /* B2 */
  }
}

static void classify_atom(const frame_t *F, int64_t i, const int8_t *species, uint32_t mask,
                          double rmsd_max, int ordering, result_t *res) {
  memset(res, 0, sizeof *res);
  res->rmsd = INFINITY;
  res->quat[0] = 1.0;
  for (int s = 0; s < NMAX; s++) res->corr[s] = -1;
  for (int s = 0; s < KMAX; s++) res->nbr[s] = -1;
  cand_t nb[TOPO_N];
  int m;
  if (ordering == 1) {                  /* topological: 18 nearest, reordered, first 14 kept */
    m = knn(F, i, TOPO_N, nb);
    if (m < 0) return;
    topo_order(m, nb, NULL);
    if (m > KMAX) m = KMAX;
  } else {
    m = knn(F, i, KMAX, nb);
    if (m < 0) return;
  }
  for (int t = 0; t < m; t++) res->nbr[t] = nb[t].j;
  double drc[3 * KMAX];
  int64_t q[3 * KMAX];
  for (int t = 0; t < m; t++) for (int d = 0; d < 3; d++) drc[3 * t + d] = nb[t].dr[d];
  ptmo_quantise(m, drc, q);

  candidate_t best;
  int have = 0;
  double best_r2 = INFINITY;
  /* collected candidates, for the tie rule */
  static __thread candidate_t *pool = NULL;
  static __thread int poolcap = 0;
  int npool = 0;

  for (int S = 0; S < NT; S++) {
    if (!(mask >> S & 1)) continue;
    const template_t *T = &TPL[S];
    const int k = T->k;
    if (m < k) continue;
    int fac[3 * 32];
    int nf = ptmo_hull(q, k, fac);
    if (nf < 0) continue;                       /* a neighbour is not a hull vertex */
    int inside = 1;
    static const int64_t zero[3] = {0, 0, 0};
    for (int f = 0; f < nf && inside; f++)
      if (sgn128(orient_exact_val(q + 3 * fac[3 * f], q + 3 * fac[3 * f + 1], q + 3 * fac[3 * f + 2], zero)) >= 0)
        inside = 0;                             /* centre must be strictly inside */
    if (!inside) continue;
    int third[KMAX][KMAX];
    build_third(k, nf, fac, third);
    for (int u = 0; u < k; u++)
      for (int v = 0; v < k; v++) {
        if (third[u][v] < 0) continue;
        uint8_t code[CODEMAX], lab[KMAX];
        int len = weinberg(k, third, u, v, code, lab);
        if (len != T->codelen) continue;
        /* all template triangulations whose fixed-start code equals this code */
        int lo = 0, hi = T->ntri;
        while (lo < hi) {
          int mid = (lo + hi) / 2;
          if (memcmp(T->codes + (size_t)T->sorted[mid] * CODEMAX, code, len) < 0) lo = mid + 1; else hi = mid;
        }
        for (int p = lo; p < T->ntri; p++) {
          int t = T->sorted[p];
          if (memcmp(T->codes + (size_t)t * CODEMAX, code, len)) break;
          /* correspondence: neighbour rank j (1..k) -> slot with the same label */
          int perm[NMAX], corr[NMAX];
          perm[0] = 0;
          for (int j = 1; j <= k; j++)
            for (int s = 1; s <= k; s++)
              if (T->labels[(size_t)t * NMAX + s] == lab[j - 1]) perm[j] = s;
          for (int j = 0; j <= k; j++) corr[perm[j]] = j;
          double v[3 * NMAX], w[3 * NMAX];
          for (int d = 0; d < 3; d++) v[d] = 0.0;
          for (int j = 1; j <= k; j++) for (int d = 0; d < 3; d++) v[3 * j + d] = nb[j - 1].dr[d];
          for (int j = 0; j <= k; j++) for (int d = 0; d < 3; d++) w[3 * j + d] = T->w[perm[j]][d];
          candidate_t cd;
          cd.S = S;
          cd.r2 = ptmo_superpose(k + 1, v, w, cd.quat, &cd.scale, NULL);
          memcpy(cd.perm, perm, sizeof perm);
          canonical_corr(T, corr, cd.cp);
          res->ncand++;
          if (npool == poolcap) { poolcap = poolcap ? 2 * poolcap : 256; pool = realloc(pool, sizeof(candidate_t) * poolcap); }
          pool[npool++] = cd;
          if (cd.r2 < best_r2) best_r2 = cd.r2;
        }
      }
  }
  /* selection with the tie rule: within TIE_R2 of the minimum, earliest template,
     then smallest canonical correspondence */
  for (int p = 0; p < npool; p++) {
    if (pool[p].r2 > best_r2 + TIE_R2) continue;
    if (!have || better(&pool[p], &best, 0)) { best = pool[p]; have = 1; }
  }
  if (!have) return;
  double rmsd = sqrt(best.r2 > 0 ? best.r2 : 0.0);
  if (rmsd > rmsd_max) return;
  const template_t *T = &TPL[best.S];
  const int k = T->k;
  res->structure = (int8_t)(best.S + 1);
  res->rmsd = rmsd;
  res->scale = best.scale;
  /* orientation reduced to the fundamental zone: the equivalent rotation Q g
     with the smallest angle (largest |w|); ties keep the earlier element */
  double bq[4] = {0}, bw = -1;
  for (int g = 0; g < T->ngroup; g++) {
    double o[4];
    quat_mul(best.quat, T->gquat[g], o);
    if (fabs(o[0]) > bw + 1e-15) { bw = fabs(o[0]); memcpy(bq, o, sizeof o); }
  }
  if (bq[0] < 0) for (int c = 0; c < 4; c++) bq[c] = -bq[c];
  memcpy(res->quat, bq, sizeof bq);
  /* correspondence as atom ids per template slot */
  res->corr[0] = (int32_t)i;
  for (int s = 1; s <= k; s++) res->corr[s] = nb[best.cp[s] - 1].j;
  /* strain (Eq. 6): both sets barycentred and scaled to mean distance 1; A^T =
     pinv(ideal) actual; then A = P U */
  {
    double act[NMAX][3], actn[NMAX][3], idl[NMAX][3];
    for (int d = 0; d < 3; d++) act[0][d] = 0.0;
    for (int s = 1; s <= k; s++) for (int d = 0; d < 3; d++) act[s][d] = nb[best.cp[s] - 1].dr[d];
    normalise(k + 1, act, actn);
    for (int s = 0; s <= k; s++) for (int d = 0; d < 3; d++) idl[s][d] = T->w[s][d];
    /* normal equations: (V^T V) A^T = V^T W */
    double VtV[3][3] = {{0}}, VtW[3][3] = {{0}};
    for (int s = 0; s <= k; s++)
      for (int a = 0; a < 3; a++) for (int b = 0; b < 3; b++) {
        VtV[a][b] += idl[s][a] * idl[s][b];
        VtW[a][b] += idl[s][a] * actn[s][b];
      }
    double inv[3][3], dV = det3(VtV);
    for (int a = 0; a < 3; a++) for (int b = 0; b < 3; b++) {
      int a1 = (b + 1) % 3, a2 = (b + 2) % 3, b1 = (a + 1) % 3, b2 = (a + 2) % 3;
      inv[a][b] = (VtV[a1][b1] * VtV[a2][b2] - VtV[a1][b2] * VtV[a2][b1]) / dV;
    }
    double At[3][3], A[9];
    for (int a = 0; a < 3; a++) for (int b = 0; b < 3; b++) {
      double s = 0;
      for (int t = 0; t < 3; t++) s += inv[a][t] * VtW[t][b];
      At[a][b] = s;
    }
    for (int a = 0; a < 3; a++) for (int b = 0; b < 3; b++) A[3 * a + b] = At[b][a];
    ptmo_polar(A, res->strain, NULL);
  }
  int32_t nid[KMAX];
  for (int t = 0; t < k; t++) nid[t] = nb[t].j;
  alloy_label(best.S, best.cp, nid, i, species, &res->alloy);
}

/* Classify the atoms listed in `atoms` (m entries) of a frame handle.  Outputs
   are indexed by list position; any output pointer may be NULL. */
int ptmo_classify(void *h, const int8_t *species, uint32_t mask, double rmsd_max, int ordering,
                  const int64_t *atoms, int64_t m,
                  int8_t *structure, int8_t *alloy, double *rmsd, double *scale,
                  double *quat, double *strain, int32_t *corr, int32_t *nbrs, int32_t *ncand) {
  if (ptmo_init()) return -1;
  const frame_t *F = h;
  for (int64_t t = 0; t < m; t++) {
    result_t r;
    classify_atom(F, atoms[t], species, mask, rmsd_max, ordering, &r);
    if (structure) structure[t] = r.structure;
    if (alloy) alloy[t] = r.alloy;
    if (rmsd) rmsd[t] = r.rmsd;
    if (scale) scale[t] = r.scale;
    if (quat) memcpy(quat + 4 * t, r.quat, sizeof r.quat);
    if (strain) memcpy(strain + 9 * t, r.strain, sizeof r.strain);
    if (corr) memcpy(corr + NMAX * t, r.corr, sizeof r.corr);
    if (nbrs) memcpy(nbrs + KMAX * t, r.nbr, sizeof r.nbr);
    if (ncand) ncand[t] = r.ncand;
  }
  return 0;
}

/* Voronoi face areas of the origin's cell among m points (Sec. 3, Eq. 5). */
int ptmo_voronoi_areas(int m, const double *v, double *area) {
  if (m < 1 || m > 64) return -1;
  double dmax = 0;
  for (int t = 0; t < m; t++) { double d2 = dot3(v + 3 * t, v + 3 * t); if (d2 > dmax) dmax = d2; }
  for (int t = 0; t < m; t++) area[t] = voronoi_face_area(m, (const double (*)[3])v, t, 10.0 * sqrt(dmax));
  return 0;
}

/* The topological order of an atom's neighbours: ids and images of the first
   min(14, m) of its 18 nearest after Eq. 5, and the 18 areas by Euclidean rank. */
int ptmo_topo_knn(void *h, int64_t atom, int32_t *ids, int32_t *imgs, double *areas) {
  const frame_t *F = h;
  cand_t nb[TOPO_N];
  int m = knn(F, atom, TOPO_N, nb);
  if (m < 0) return m;
  topo_order(m, nb, areas);
  int k = m > KMAX ? KMAX : m;
  for (int t = 0; t < k; t++) { ids[t] = nb[t].j; for (int c = 0; c < 3; c++) imgs[3 * t + c] = nb[t].n[c]; }
  return k;
}
