/*
 * oracle.c -- plain FP64 CPU oracle for the AO/MO "vgl" path and its adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline
 * leg of the benchmark are the only callers.  It shares no code, header,
 * table or helper with the CUDA library, and the CUDA library never calls it.
 *
 * What it computes, written from the definitions (QMCkl paper, Sec. 3):
 *
 *   chi_n(r)  = M_n R_s(r) P_abc(r)                        (Eq. 1)
 *   R_s(r)    = N_s sum_k a_ks f_ks exp(-gamma_ks |r-R_A|^2)  (Eq. 2, p=2, n_s=0)
 *   P_abc(r)  = (x-X_A)^a (y-Y_A)^b (z-Z_A)^c               (Eq. 4)
 *   primitive k is evaluated only if gamma_ks |r-R_A|^2 < T  (Eq. 3), where
 *   T = (B-1) ln 2 for B precision bits (T = +inf: unscreened)
 *   phi_n, grad phi_n, lap phi_n = sum_k C_nk (chi_k, grad chi_k, lap chi_k)
 *                                                            (Eqs. 5-7)
 *
 * Derivatives are taken primitive by primitive.  Because
 * exp(-g r^2) = exp(-g x^2) exp(-g y^2) exp(-g z^2), a Cartesian primitive
 * factorises into three 1-D functions x^a exp(-g x^2); the m-th derivative of
 * that 1-D function is q_m(x) exp(-g x^2) with q_0 = x^a and
 * q_{m+1} = q_m' - 2 g x q_m.  Any mixed derivative d^i/dx d^j/dy d^k/dz of
 * the primitive is q_i(x) q_j(y) q_k(z) exp(-g r^2).
 *
 * Sums over AOs (the MO contraction) and over points (the adjoint) use the
 * compensated dot product "Dot2" of Ogita, Rump and Oishi (SIAM J. Sci.
 * Comput. 26, 2005): TwoProduct via fma plus TwoSum, which returns the result
 * as if computed in twice the working precision.  Compile with
 * -ffp-contract=off so that the error-free transformations stay exact.
 *
 * Every output array is caller-owned.  Functions return 0 on success and a
 * negative value on bad arguments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int64_t nucl_num;
  const double* nucl_coord;       /* [nucl][3] */
  int64_t shell_num;
  const int64_t* shell_nucleus;   /* [shell] */
  const int32_t* shell_ang_mom;   /* [shell] */
  const int64_t* shell_prim_num;  /* [shell]; primitives stored shell-major */
  const double* shell_factor;     /* [shell] N_s */
  int64_t prim_num;
  const double* exponent;         /* [prim] gamma */
  const double* coefficient;      /* [prim] a */
  const double* prim_factor;      /* [prim] f */
  int64_t ao_num;
  const double* ao_factor;        /* [ao] M_n */
} oracle_basis_t;

/* ---------------------------------------------------------------- Dot2 --- */
typedef struct { double p, s; } dot2_t;

static void dot2_add(dot2_t* acc, double x, double y) {
  double h = x * y;
  double r = fma(x, y, -h);          /* TwoProduct: x*y = h + r exactly */
  double p = acc->p + h;             /* TwoSum(acc->p, h) = p + q */
  double z = p - acc->p;
  double q = (acc->p - (p - z)) + (h - z);
  acc->p = p;
  acc->s += q + r;
}
static double dot2_value(const dot2_t* acc) { return acc->p + acc->s; }

/* --------------------------------------------- 1-D derivative factors --- */
#define QDEG 8   /* a <= 3 and up to 3 derivatives: degree <= 6 */
#define QORD 4   /* derivative orders 0..3 */

/* q[m][i]: coefficient of x^i in the m-th derivative factor of x^a e^{-g x^2} */
static void deriv_factors(int a, double g, double q[QORD][QDEG]) {
  memset(q, 0, sizeof(double) * QORD * QDEG);
  q[0][a] = 1.0;
  for (int m = 0; m + 1 < QORD; ++m)
    for (int i = 0; i < QDEG; ++i) {
      double c = q[m][i];
      if (c == 0.0) continue;
      if (i > 0) q[m + 1][i - 1] += (double)i * c;       /* derivative of x^i */
      if (i + 1 < QDEG) q[m + 1][i + 1] += -2.0 * g * c; /* -2 g x times x^i */
    }
}

static double poly_value(const double* q, double x) {
  double s = 0.0, xp = 1.0;
  for (int i = 0; i < QDEG; ++i) { s += q[i] * xp; xp *= x; }
  return s;
}

/* sum_i |q_i| |x|^i : the size of the terms whose sum poly_value returns */
static double poly_size(const double* q, double x) {
  double s = 0.0, xp = 1.0, ax = fabs(x);
  for (int i = 0; i < QDEG; ++i) { s += fabs(q[i]) * xp; xp *= ax; }
  return s;
}

/* (a,b,c) of the j-th Cartesian component of a shell of momentum l,
   lexicographic by descending a then descending b. */
static void cart_powers(int l, int j, int* a, int* b, int* c) {
  int n = 0;
  for (int aa = l; aa >= 0; --aa)
    for (int bb = l - aa; bb >= 0; --bb) {
      if (n == j) { *a = aa; *b = bb; *c = l - aa - bb; return; }
      ++n;
    }
  *a = *b = *c = -1;
}

static int check_basis(const oracle_basis_t* b) {
  if (!b || b->shell_num < 0 || b->nucl_num < 0 || b->ao_num < 0) return -1;
  int64_t prim = 0, ao = 0;
  for (int64_t s = 0; s < b->shell_num; ++s) {
    int l = b->shell_ang_mom[s];
    if (l < 0 || l > 3) return -2;
    if (b->shell_nucleus[s] < 0 || b->shell_nucleus[s] >= b->nucl_num) return -3;
    prim += b->shell_prim_num[s];
    ao += (l + 1) * (l + 2) / 2;
  }
  if (prim != b->prim_num || ao != b->ao_num) return -4;
  return 0;
}

double oracle_threshold_bits(int bits) { return (double)(bits - 1) * log(2.0); }
double oracle_threshold_eps(double eps) { return -log(eps); }

/*
 * Mixed derivatives of every AO at one point.  deriv(ix,iy,iz) for the
 * orders listed in `orders` ([norder][3]) -> out[o][ao] and size[o][ao]
 * (size: the same sum with every term replaced by its absolute value).
 */
static void ao_derivs_point(const oracle_basis_t* b, double T, const double* r,
                            int norder, const int (*orders)[3],
                            double* out, double* size) {
  memset(out, 0, sizeof(double) * (size_t)norder * (size_t)b->ao_num);
  if (size) memset(size, 0, sizeof(double) * (size_t)norder * (size_t)b->ao_num);
  int64_t prim0 = 0, ao0 = 0;
  for (int64_t s = 0; s < b->shell_num; ++s) {
    const int l = b->shell_ang_mom[s];
    const int ncart = (l + 1) * (l + 2) / 2;
    const double* R = b->nucl_coord + 3 * b->shell_nucleus[s];
    const double dx = r[0] - R[0], dy = r[1] - R[1], dz = r[2] - R[2];
    const double r2 = dx * dx + dy * dy + dz * dz;
    for (int64_t k = prim0; k < prim0 + b->shell_prim_num[s]; ++k) {
      const double g = b->exponent[k];
      if (!(g * r2 < T)) continue;                       /* Eq. 3 */
      const double e = exp(-g * r2);
      const double cf = b->shell_factor[s] * b->coefficient[k] * b->prim_factor[k];
      for (int j = 0; j < ncart; ++j) {
        int a, bb, c;
        cart_powers(l, j, &a, &bb, &c);
        double qx[QORD][QDEG], qy[QORD][QDEG], qz[QORD][QDEG];
        deriv_factors(a, g, qx);
        deriv_factors(bb, g, qy);
        deriv_factors(c, g, qz);
        const double w = b->ao_factor[ao0 + j] * cf * e;
        for (int o = 0; o < norder; ++o) {
          const int ix = orders[o][0], iy = orders[o][1], iz = orders[o][2];
          out[(size_t)o * b->ao_num + ao0 + j] +=
              w * poly_value(qx[ix], dx) * poly_value(qy[iy], dy) * poly_value(qz[iz], dz);
          if (size)
            size[(size_t)o * b->ao_num + ao0 + j] +=
                fabs(w) * poly_size(qx[ix], dx) * poly_size(qy[iy], dy) * poly_size(qz[iz], dz);
        }
      }
    }
    prim0 += b->shell_prim_num[s];
    ao0 += ncart;
  }
}

/* derivative orders: value, d/dx, d/dy, d/dz, then d2/dx2, d2/dy2, d2/dz2 */
static const int VGL_ORDERS[7][3] = {
  {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2}};

/*
 * AO values, gradients and Laplacians at `n` points.
 * coord [n][3]; vgl [n][5][ao] (v, dx, dy, dz, lap); mag (optional) the
 * term-wise absolute size of each entry, for cancellation-aware error bars.
 */
int oracle_ao_vgl(const oracle_basis_t* b, double T, int64_t n, const double* coord,
                  double* vgl, double* mag) {
  int rc = check_basis(b);
  if (rc) return rc;
  const int64_t na = b->ao_num;
  double* d = (double*)malloc(sizeof(double) * 7 * (size_t)(na ? na : 1));
  double* z = (double*)malloc(sizeof(double) * 7 * (size_t)(na ? na : 1));
  if (!d || !z) { free(d); free(z); return -9; }
  for (int64_t p = 0; p < n; ++p) {
    ao_derivs_point(b, T, coord + 3 * p, 7, VGL_ORDERS, d, z);
    double* o = vgl + (size_t)p * 5 * na;
    double* m = mag ? mag + (size_t)p * 5 * na : NULL;
    for (int64_t k = 0; k < na; ++k) {
      for (int c = 0; c < 4; ++c) o[c * na + k] = d[c * na + k];
      o[4 * na + k] = d[4 * na + k] + d[5 * na + k] + d[6 * na + k];
      if (m) {
        for (int c = 0; c < 4; ++c) m[c * na + k] = z[c * na + k];
        m[4 * na + k] = z[4 * na + k] + z[5 * na + k] + z[6 * na + k];
      }
    }
  }
  free(d);
  free(z);
  return 0;
}

/*
 * MO vgl from AO vgl (Eqs. 5-7): mo[p][c][i] = sum_k C[i][k] ao[p][c][k].
 * mo_mag (optional) = sum_k |C[i][k]| ao_mag[p][c][k] (needs ao_mag).
 */
int oracle_mo_vgl(int64_t ao_num, int64_t mo_num, const double* C, int64_t n,
                  const double* ao_vgl, const double* ao_mag, double* mo, double* mo_mag) {
  if (ao_num < 0 || mo_num < 0 || n < 0) return -1;
  if (mo_mag && !ao_mag) return -1;
  for (int64_t p = 0; p < n; ++p)
    for (int c = 0; c < 5; ++c) {
      const double* a = ao_vgl + ((size_t)p * 5 + c) * ao_num;
      const double* am = ao_mag ? ao_mag + ((size_t)p * 5 + c) * ao_num : NULL;
      for (int64_t i = 0; i < mo_num; ++i) {
        const double* ci = C + (size_t)i * ao_num;
        dot2_t acc = {0.0, 0.0};
        double sz = 0.0;
        for (int64_t k = 0; k < ao_num; ++k) {
          dot2_add(&acc, ci[k], a[k]);
          if (mo_mag) sz += fabs(ci[k]) * am[k];
        }
        mo[((size_t)p * 5 + c) * mo_num + i] = dot2_value(&acc);
        if (mo_mag) mo_mag[((size_t)p * 5 + c) * mo_num + i] = sz;
      }
    }
  return 0;
}

/* AO then MO vgl at n points, one point at a time (no n*5*ao buffer). */
int oracle_mo_vgl_points(const oracle_basis_t* b, double T, int64_t mo_num, const double* C,
                         int64_t n, const double* coord, double* mo, double* mo_mag) {
  int rc = check_basis(b);
  if (rc) return rc;
  const int64_t na = b->ao_num;
  double* a = (double*)malloc(sizeof(double) * 5 * (size_t)(na ? na : 1));
  double* am = (double*)malloc(sizeof(double) * 5 * (size_t)(na ? na : 1));
  if (!a || !am) { free(a); free(am); return -9; }
  for (int64_t p = 0; p < n; ++p) {
    rc = oracle_ao_vgl(b, T, 1, coord + 3 * p, a, am);
    if (!rc)
      rc = oracle_mo_vgl(na, mo_num, C, 1, a, am, mo + (size_t)p * 5 * mo_num,
                         mo_mag ? mo_mag + (size_t)p * 5 * mo_num : NULL);
    if (rc) break;
  }
  free(a);
  free(am);
  return rc;
}

/* orders for the adjoint: all mixed derivatives of total order <= 3 */
static int order_index(int ix, int iy, int iz) {
  /* enumerate (ix,iy,iz) with ix+iy+iz <= 3 in a fixed order */
  int n = 0;
  for (int t = 0; t <= 3; ++t)
    for (int a = t; a >= 0; --a)
      for (int b2 = t - a; b2 >= 0; --b2) {
        if (a == ix && b2 == iy && t - a - b2 == iz) return n;
        ++n;
      }
  return -1;
}
static int ADJ_ORDERS[20][3];
static int adj_orders_ready = 0;
static void init_adj_orders(void) {
  if (adj_orders_ready) return;
  int n = 0;
  for (int t = 0; t <= 3; ++t)
    for (int a = t; a >= 0; --a)
      for (int b2 = t - a; b2 >= 0; --b2) {
        ADJ_ORDERS[n][0] = a; ADJ_ORDERS[n][1] = b2; ADJ_ORDERS[n][2] = t - a - b2;
        ++n;
      }
  adj_orders_ready = 1;
}

/*
 * Adjoint of L = sum_{p,c,i} W[p][c][i] mo[p][c][i] (mo from Eqs. 5-7).
 *   dC[i][k] = sum_{p,c} W[p][c][i] ao[p][c][k]
 *   Abar[p][c][k] = sum_i W[p][c][i] C[i][k]
 *   dR[A][j] = sum_p sum_{k on A} sum_c Abar[p][c][k] d ao[p][c][k] / dR_Aj
 * and since an AO on A depends on r - R_A only, d/dR_Aj = -d/dr_j:
 *   c = value -> -d_j chi; c = d_i -> -d_j d_i chi; c = lap -> -d_j lap chi.
 * W [n][5][mo]; dC [mo][ao]; dR [nucl][3].  Either output may be NULL.
 * dC_size, dR_size (optional, same shapes): the same sums with every factor
 * replaced by the absolute size of its terms (|W|, sum_i |W||C| for Abar,
 * and the term-wise size of each AO derivative): the scale against which a
 * rounding error of the sum is measured.
 */
int oracle_adjoint(const oracle_basis_t* b, double T, int64_t mo_num, const double* C,
                   int64_t n, const double* coord, const double* W,
                   double* dC, double* dR, double* dC_size, double* dR_size) {
  int rc = check_basis(b);
  if (rc) return rc;
  init_adj_orders();
  const int64_t na = b->ao_num;
  double* d = (double*)malloc(sizeof(double) * 20 * (size_t)(na ? na : 1));
  double* z = (double*)malloc(sizeof(double) * 20 * (size_t)(na ? na : 1));
  double* abar = (double*)malloc(sizeof(double) * 5 * (size_t)(na ? na : 1));
  double* abar_sz = (double*)malloc(sizeof(double) * 5 * (size_t)(na ? na : 1));
  dot2_t* accC = dC ? (dot2_t*)calloc((size_t)mo_num * (na ? na : 1), sizeof(dot2_t)) : NULL;
  dot2_t* accR = (dot2_t*)calloc((size_t)3 * (b->nucl_num ? b->nucl_num : 1), sizeof(dot2_t));
  int64_t* ao_nuc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(na ? na : 1));
  if (!d || !z || !abar || !abar_sz || (dC && !accC) || !accR || !ao_nuc) {
    free(d); free(z); free(abar); free(abar_sz); free(accC); free(accR); free(ao_nuc);
    return -9;
  }
  if (dC_size) memset(dC_size, 0, sizeof(double) * (size_t)mo_num * na);
  if (dR_size) memset(dR_size, 0, sizeof(double) * 3 * (size_t)b->nucl_num);
  {
    int64_t ao0 = 0;
    for (int64_t s = 0; s < b->shell_num; ++s) {
      int l = b->shell_ang_mom[s];
      for (int j = 0; j < (l + 1) * (l + 2) / 2; ++j) ao_nuc[ao0 + j] = b->shell_nucleus[s];
      ao0 += (l + 1) * (l + 2) / 2;
    }
  }
  for (int64_t p = 0; p < n; ++p) {
    ao_derivs_point(b, T, coord + 3 * p, 20, (const int (*)[3])ADJ_ORDERS, d, z);
    const double* w = W + (size_t)p * 5 * mo_num;
    /* AO vgl at this point, component c, AO k: from the derivative table */
#define DV(ix, iy, iz, k) d[(size_t)order_index(ix, iy, iz) * na + (k)]
#define DZ(ix, iy, iz, k) z[(size_t)order_index(ix, iy, iz) * na + (k)]
    for (int64_t k = 0; k < na; ++k) {
      double ao_c[5], ao_z[5];
      ao_c[0] = DV(0, 0, 0, k);
      ao_c[1] = DV(1, 0, 0, k);
      ao_c[2] = DV(0, 1, 0, k);
      ao_c[3] = DV(0, 0, 1, k);
      ao_c[4] = DV(2, 0, 0, k) + DV(0, 2, 0, k) + DV(0, 0, 2, k);
      ao_z[0] = DZ(0, 0, 0, k);
      ao_z[1] = DZ(1, 0, 0, k);
      ao_z[2] = DZ(0, 1, 0, k);
      ao_z[3] = DZ(0, 0, 1, k);
      ao_z[4] = DZ(2, 0, 0, k) + DZ(0, 2, 0, k) + DZ(0, 0, 2, k);
      for (int c = 0; c < 5; ++c) {
        dot2_t acc = {0.0, 0.0};
        double asz = 0.0;
        for (int64_t i = 0; i < mo_num; ++i) {
          const double wv = w[(size_t)c * mo_num + i];
          dot2_add(&acc, wv, C[(size_t)i * na + k]);
          asz += fabs(wv) * fabs(C[(size_t)i * na + k]);
          if (accC) dot2_add(&accC[(size_t)i * na + k], wv, ao_c[c]);
          if (dC_size) dC_size[(size_t)i * na + k] += fabs(wv) * ao_z[c];
        }
        abar[(size_t)c * na + k] = dot2_value(&acc);
        abar_sz[(size_t)c * na + k] = asz;
      }
    }
    if (dR) {
      for (int64_t k = 0; k < na; ++k) {
        const int64_t A = ao_nuc[k];
        for (int j = 0; j < 3; ++j) {
          const int e[3] = {j == 0, j == 1, j == 2};
          /* d_j of each vgl component */
          double g[5];
          g[0] = DV(e[0], e[1], e[2], k);
          g[1] = DV(1 + e[0], e[1], e[2], k);
          g[2] = DV(e[0], 1 + e[1], e[2], k);
          g[3] = DV(e[0], e[1], 1 + e[2], k);
          g[4] = DV(2 + e[0], e[1], e[2], k) + DV(e[0], 2 + e[1], e[2], k) +
                 DV(e[0], e[1], 2 + e[2], k);
          for (int c = 0; c < 5; ++c) dot2_add(&accR[3 * A + j], -abar[(size_t)c * na + k], g[c]);
          if (dR_size) {
            double gz[5];
            gz[0] = DZ(e[0], e[1], e[2], k);
            gz[1] = DZ(1 + e[0], e[1], e[2], k);
            gz[2] = DZ(e[0], 1 + e[1], e[2], k);
            gz[3] = DZ(e[0], e[1], 1 + e[2], k);
            gz[4] = DZ(2 + e[0], e[1], e[2], k) + DZ(e[0], 2 + e[1], e[2], k) +
                    DZ(e[0], e[1], 2 + e[2], k);
            for (int c = 0; c < 5; ++c) dR_size[3 * A + j] += abar_sz[(size_t)c * na + k] * gz[c];
          }
        }
      }
    }
#undef DV
#undef DZ
  }
  if (dC)
    for (size_t t = 0; t < (size_t)mo_num * na; ++t) dC[t] = dot2_value(&accC[t]);
  if (dR)
    for (int64_t t = 0; t < 3 * b->nucl_num; ++t) dR[t] = dot2_value(&accR[t]);
  free(d); free(z); free(abar); free(abar_sz); free(accC); free(accR); free(ao_nuc);
  return 0;
}

/*
 * Screening work counts at n points: counts[0] = (point, shell) pairs with
 * at least one primitive passing Eq. 3, counts[1] = primitives evaluated,
 * counts[2] = (point, AO) pairs inside a surviving shell.
 */
int oracle_screen_counts(const oracle_basis_t* b, double T, int64_t n, const double* coord,
                         int64_t* counts) {
  int rc = check_basis(b);
  if (rc) return rc;
  counts[0] = counts[1] = counts[2] = 0;
  for (int64_t p = 0; p < n; ++p) {
    const double* r = coord + 3 * p;
    int64_t prim0 = 0;
    for (int64_t s = 0; s < b->shell_num; ++s) {
      const double* R = b->nucl_coord + 3 * b->shell_nucleus[s];
      const double dx = r[0] - R[0], dy = r[1] - R[1], dz = r[2] - R[2];
      const double r2 = dx * dx + dy * dy + dz * dz;
      int64_t np = 0;
      for (int64_t k = prim0; k < prim0 + b->shell_prim_num[s]; ++k)
        if (b->exponent[k] * r2 < T) ++np;
      if (np) {
        int l = b->shell_ang_mom[s];
        counts[0] += 1;
        counts[1] += np;
        counts[2] += (l + 1) * (l + 2) / 2;
      }
      prim0 += b->shell_prim_num[s];
    }
  }
  return 0;
}
