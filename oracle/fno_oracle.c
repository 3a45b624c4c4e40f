/*
 * fno_oracle.c -- plain, slow FP64 CPU oracle of the 4-D spectral FNO block
 * and its gradient.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check of the package
 * entry file and the CPU-baseline / reference legs of bench.py load this
 * library.  The CUDA product path never calls it and shares no code, table or
 * header with it.
 *
 * What it computes (the FNO block of Alg. 2, Sec. IV-C of the paper, with the
 * bypass 1x1 linear + bias of the original FNO that Sec. IV-C says the
 * architecture follows, and the nonlinearity sigma of Alg. 1 taken as GELU):
 *
 *   theta_j(p) = 2 pi (kx x/Nx + ky y/Ny + kz z/Nz + kt t/Nt)
 *   Xh[b,i,j]  = sum_p X[b,i,p] exp(-i theta_j(p))        forward DFT F, truncation S
 *   Yh[b,o,j]  = sum_i Xh[b,i,j] W[i,o,j]                 spectral convolution (einsum of Alg. 2)
 *   S[b,o,p]   = (1/N) sum_j c(kt_j) Re(Yh[b,o,j] exp(+i theta_j(p)))   padding S^T, inverse F^T
 *   A[b,o,p]   = S[b,o,p] + sum_i X[b,i,p] Wl[i,o] + bias[o]
 *   Z          = GELU(A) = A (1 + erf(A/sqrt 2)) / 2
 *
 * Kept set: kx in {0..mx-1} U {-mx..-1}, stored index jx < mx -> kx = jx,
 * jx >= mx -> kx = jx - 2 mx (same for y and z); kt in {0..mt-1} (the real
 * half spectrum of the last, contiguous axis).  c(kt) = 1 at kt = 0 and at the
 * Nyquist bin kt = Nt/2 (Nt even), 2 otherwise, so S is the real field whose
 * Hermitian-completed spectrum is the kept one.  The forward transform is
 * unnormalised and the inverse carries 1/N ("backward" normalisation).
 *
 * Gradient (derived by differentiating the five lines above in the real and
 * imaginary parts; complex gradients are dL/dRe + i dL/dIm):
 *   dA = dZ GELU'(A);  db[o] = sum dA;  dWl[i,o] = sum X[b,i,p] dA[b,o,p]
 *   G[b,o,j]  = (c(kt_j)/N) sum_p dA[b,o,p] exp(-i theta_j(p))
 *   dW[i,o,j] = sum_b conj(Xh[b,i,j]) G[b,o,j]
 *   GXh[b,i,j]= sum_o conj(W[i,o,j]) G[b,o,j]
 *   dX[b,i,p] = sum_j Re(GXh[b,i,j] exp(+i theta_j(p))) + sum_o Wl[i,o] dA[b,o,p]
 *
 * Evaluation: separable direct summation (no FFT), forward axis order
 * t -> z -> y -> x as in Alg. 2 (the non-partitioned y,z,t first, x last),
 * the inverse in the reverse order.  Every phase is taken from per-axis FP64
 * tables of exp(2 pi i r/N) indexed by the exact integer residue r = k n mod N.
 * The brute-force routines evaluate the full 4-D sums literally with their own
 * cos/sin calls, for tiny shapes.
 *
 * Around the blocks (Alg. 1): the encoder and decoder pointwise 1x1 layers
 * with sigma, the mean-squared-error loss, and the Adam update of a training
 * step, at the end of this file.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI 6.283185307179586476925286766559005768

/* Mutation hooks for the pin tests: a test build defines ORACLE_MUTANT = k to
 * plant one known slip (1 stored-index map off by one, 2 dropped c(kt),
 * 3 wrong sign of the t exponent, 4 missing 1/N, 5 transposed W_l in the
 * forward, 6 conjugate dropped in dW, 7 GELU' without its second term,
 * 8 bias dropped in the pointwise layer, 9 loss gradient without its factor 2,
 * 10 pointwise sigma' taken at sigma(A) instead of A, 11 Adam's second moment
 * fed g instead of g^2) and checks that some pin fails.  The oracle itself is
 * built with 0. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#define MUT(k) (ORACLE_MUTANT == (k))

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2 };

typedef struct {
  int64_t B, Ci, Co, Nx, Ny, Nz, Nt, mx, my, mz, mt;
  int64_t Jx, Jy, Jz, Jt; /* stored mode counts per axis */
  int64_t Ng;             /* grid points per channel */
  int64_t Mk;             /* kept modes per channel */
} dims_t;

/* dims array layout: B, Ci, Co, Nx, Ny, Nz, Nt, mx, my, mz, mt */
static int dims_from(const int64_t* a, dims_t* d) {
  if (!a) return ORC_EINVAL;
  d->B = a[0]; d->Ci = a[1]; d->Co = a[2];
  d->Nx = a[3]; d->Ny = a[4]; d->Nz = a[5]; d->Nt = a[6];
  d->mx = a[7]; d->my = a[8]; d->mz = a[9]; d->mt = a[10];
  for (int q = 0; q < 11; ++q)
    if (a[q] <= 0) return ORC_EINVAL;
  if (2 * d->mx > d->Nx || 2 * d->my > d->Ny || 2 * d->mz > d->Nz) return ORC_EINVAL;
  if (d->mt > d->Nt / 2 + 1) return ORC_EINVAL;
  d->Jx = 2 * d->mx; d->Jy = 2 * d->my; d->Jz = 2 * d->mz; d->Jt = d->mt;
  d->Ng = d->Nx * d->Ny * d->Nz * d->Nt;
  d->Mk = d->Jx * d->Jy * d->Jz * d->Jt;
  return ORC_OK;
}

static int64_t rmod(int64_t a, int64_t n) {
  int64_t r = a % n;
  return r < 0 ? r + n : r;
}

/* signed frequency of stored index j on a symmetric axis with m kept per side */
static int64_t kfreq(int64_t j, int64_t m) { return j < m ? j : j - 2 * m + (MUT(1) ? 1 : 0); }

/* weight of a half-spectrum bin in the real synthesis */
static double cweight(int64_t kt, int64_t Nt) {
  if (MUT(2)) return 1.0;
  if (kt == 0) return 1.0;
  if (Nt % 2 == 0 && 2 * kt == Nt) return 1.0;
  return 2.0;
}

/* ---- per-axis tables -------------------------------------------------- */

typedef struct {
  int64_t n;
  double* c; /* cos(2 pi r / n) */
  double* s; /* sin(2 pi r / n) */
} trig_t;

typedef struct {
  trig_t x, y, z, t;
  int64_t *kx, *ky, *kz, *kt;
} tables_t;

static int trig_make(trig_t* tg, int64_t n) {
  tg->n = n;
  tg->c = (double*)malloc(sizeof(double) * (size_t)n);
  tg->s = (double*)malloc(sizeof(double) * (size_t)n);
  if (!tg->c || !tg->s) return ORC_ENOMEM;
  for (int64_t r = 0; r < n; ++r) {
    double a = TWO_PI * (double)r / (double)n;
    tg->c[r] = cos(a);
    tg->s[r] = sin(a);
  }
  return ORC_OK;
}

static void trig_free(trig_t* tg) { free(tg->c); free(tg->s); tg->c = tg->s = NULL; }

static void tables_free(tables_t* T) {
  trig_free(&T->x); trig_free(&T->y); trig_free(&T->z); trig_free(&T->t);
  free(T->kx); free(T->ky); free(T->kz); free(T->kt);
  memset(T, 0, sizeof(*T));
}

static int tables_make(const dims_t* d, tables_t* T) {
  memset(T, 0, sizeof(*T));
  int rc = 0;
  rc |= trig_make(&T->x, d->Nx);
  rc |= trig_make(&T->y, d->Ny);
  rc |= trig_make(&T->z, d->Nz);
  rc |= trig_make(&T->t, d->Nt);
  T->kx = (int64_t*)malloc(sizeof(int64_t) * (size_t)d->Jx);
  T->ky = (int64_t*)malloc(sizeof(int64_t) * (size_t)d->Jy);
  T->kz = (int64_t*)malloc(sizeof(int64_t) * (size_t)d->Jz);
  T->kt = (int64_t*)malloc(sizeof(int64_t) * (size_t)d->Jt);
  if (rc || !T->kx || !T->ky || !T->kz || !T->kt) { tables_free(T); return ORC_ENOMEM; }
  for (int64_t j = 0; j < d->Jx; ++j) T->kx[j] = kfreq(j, d->mx);
  for (int64_t j = 0; j < d->Jy; ++j) T->ky[j] = kfreq(j, d->my);
  for (int64_t j = 0; j < d->Jz; ++j) T->kz[j] = kfreq(j, d->mz);
  for (int64_t j = 0; j < d->Jt; ++j) T->kt[j] = j;
  return ORC_OK;
}

/* ---- one axis of the separable transforms ------------------------------ */

/* Forward along one axis of a complex array (mode index on the output):
 *   out[o][j][i] = sum_{q<n} in[o][q][i] exp(-2 pi i k[j] q / n)            */
static void axis_forward(const double* in, double* out, int64_t outer, int64_t n, int64_t J,
                         int64_t inner, const int64_t* k, const trig_t* tg) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t o = 0; o < outer; ++o) {
    for (int64_t j = 0; j < J; ++j) {
      double* dst = out + 2 * ((o * J + j) * inner);
      for (int64_t i = 0; i < inner; ++i) { dst[2 * i] = 0.0; dst[2 * i + 1] = 0.0; }
      for (int64_t q = 0; q < n; ++q) {
        int64_t r = rmod(k[j] * q, n);
        double c = tg->c[r], s = -tg->s[r];
        const double* src = in + 2 * ((o * n + q) * inner);
        for (int64_t i = 0; i < inner; ++i) {
          double a = src[2 * i], b = src[2 * i + 1];
          dst[2 * i] += a * c - b * s;
          dst[2 * i + 1] += a * s + b * c;
        }
      }
    }
  }
}

/* Inverse along one axis (mode index on the input), zero padding implied:
 *   out[o][q][i] = sum_{j<J} in[o][j][i] exp(+2 pi i k[j] q / n)            */
static void axis_inverse(const double* in, double* out, int64_t outer, int64_t J, int64_t n,
                         int64_t inner, const int64_t* k, const trig_t* tg) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t o = 0; o < outer; ++o) {
    for (int64_t q = 0; q < n; ++q) {
      double* dst = out + 2 * ((o * n + q) * inner);
      for (int64_t i = 0; i < inner; ++i) { dst[2 * i] = 0.0; dst[2 * i + 1] = 0.0; }
      for (int64_t j = 0; j < J; ++j) {
        int64_t r = rmod(k[j] * q, n);
        double c = tg->c[r], s = tg->s[r];
        const double* src = in + 2 * ((o * J + j) * inner);
        for (int64_t i = 0; i < inner; ++i) {
          double a = src[2 * i], b = src[2 * i + 1];
          dst[2 * i] += a * c - b * s;
          dst[2 * i + 1] += a * s + b * c;
        }
      }
    }
  }
}

/* ---- one channel: spectrum and synthesis ------------------------------- */

typedef struct {
  double *p1, *p2, *p3; /* stage buffers, sized for the largest use */
} work_t;

static int work_make(const dims_t* d, work_t* w) {
  size_t n1 = (size_t)(d->Nx * d->Ny * d->Nz * d->Jt) * 2;
  size_t n2 = (size_t)(d->Nx * d->Ny * d->Jz * d->Jt) * 2;
  size_t n3 = (size_t)(d->Nx * d->Jy * d->Jz * d->Jt) * 2;
  w->p1 = (double*)malloc(sizeof(double) * n1);
  w->p2 = (double*)malloc(sizeof(double) * n2);
  w->p3 = (double*)malloc(sizeof(double) * n3);
  if (!w->p1 || !w->p2 || !w->p3) {
    free(w->p1); free(w->p2); free(w->p3);
    return ORC_ENOMEM;
  }
  return ORC_OK;
}

static void work_free(work_t* w) { free(w->p1); free(w->p2); free(w->p3); }

/* fh[jx][jy][jz][jt] = sum_{x,y,z,t} f[x][y][z][t] exp(-i theta_j); when
 * adjoint_scale is set every mode is then multiplied by c(kt)/N (the G of the
 * gradient). Axis order t, z, y, x. */
static void spectrum_one(const dims_t* d, const tables_t* T, const double* f, double* fh,
                         int adjoint_scale, work_t* w) {
  const int64_t rows = d->Nx * d->Ny * d->Nz;
  const int64_t Nt = d->Nt, Jt = d->Jt;
  double* p1 = w->p1;
  /* t: real -> complex half spectrum */
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < rows; ++r) {
    const double* src = f + r * Nt;
    double* dst = p1 + 2 * r * Jt;
    for (int64_t jt = 0; jt < Jt; ++jt) {
      double re = 0.0, im = 0.0;
      for (int64_t t = 0; t < Nt; ++t) {
        int64_t q = rmod(T->kt[jt] * t, Nt);
        re += src[t] * T->t.c[q];
        im -= (MUT(3) ? -1.0 : 1.0) * src[t] * T->t.s[q];
      }
      dst[2 * jt] = re;
      dst[2 * jt + 1] = im;
    }
  }
  /* z, y, x */
  axis_forward(p1, w->p2, d->Nx * d->Ny, d->Nz, d->Jz, Jt, T->kz, &T->z);
  axis_forward(w->p2, w->p3, d->Nx, d->Ny, d->Jy, d->Jz * Jt, T->ky, &T->y);
  axis_forward(w->p3, fh, 1, d->Nx, d->Jx, d->Jy * d->Jz * Jt, T->kx, &T->x);
  if (adjoint_scale) {
    const double invN = 1.0 / (double)d->Ng;
    for (int64_t m = 0; m < d->Mk; ++m) {
      double s = cweight(T->kt[m % Jt], Nt) * invN;
      fh[2 * m] *= s;
      fh[2 * m + 1] *= s;
    }
  }
}

/* f[x][y][z][t] = sum_j wgt(kt) Re(fh_j exp(+i theta_j(p))); wgt = c(kt)/N
 * when scaled (the block's inverse), 1 otherwise (the adjoint of the
 * unnormalised forward transform).  Axis order x, y, z, t. */
static void synthesis_one(const dims_t* d, const tables_t* T, const double* fh, double* f,
                          int scaled, work_t* w) {
  const int64_t Nt = d->Nt, Jt = d->Jt;
  axis_inverse(fh, w->p3, 1, d->Jx, d->Nx, d->Jy * d->Jz * Jt, T->kx, &T->x);
  axis_inverse(w->p3, w->p2, d->Nx, d->Jy, d->Ny, d->Jz * Jt, T->ky, &T->y);
  axis_inverse(w->p2, w->p1, d->Nx * d->Ny, d->Jz, d->Nz, Jt, T->kz, &T->z);
  const int64_t rows = d->Nx * d->Ny * d->Nz;
  const double invN = MUT(4) ? 1.0 : 1.0 / (double)d->Ng;
  const double* q1 = w->p1;
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < rows; ++r) {
    const double* src = q1 + 2 * r * Jt;
    double* dst = f + r * Nt;
    for (int64_t t = 0; t < Nt; ++t) {
      double acc = 0.0;
      for (int64_t jt = 0; jt < Jt; ++jt) {
        int64_t q = rmod(T->kt[jt] * t, Nt);
        double wgt = scaled ? cweight(T->kt[jt], Nt) * invN : 1.0;
        acc += wgt * (src[2 * jt] * T->t.c[q] - src[2 * jt + 1] * T->t.s[q]);
      }
      dst[t] = acc;
    }
  }
}

/* the same synthesis evaluated at single grid points (x,y,z,t) */
static double synthesis_point(const dims_t* d, const tables_t* T, const double* fh,
                              const int64_t* p, int scaled) {
  const int64_t x = p[0], y = p[1], z = p[2], t = p[3];
  const double invN = 1.0 / (double)d->Ng;
  double accr = 0.0;
  for (int64_t jx = 0; jx < d->Jx; ++jx) {
    int64_t rx = rmod(T->kx[jx] * x, d->Nx);
    double cxr = T->x.c[rx], cxi = T->x.s[rx];
    for (int64_t jy = 0; jy < d->Jy; ++jy) {
      int64_t ry = rmod(T->ky[jy] * y, d->Ny);
      double cyr = T->y.c[ry], cyi = T->y.s[ry];
      double exyr = cxr * cyr - cxi * cyi, exyi = cxr * cyi + cxi * cyr;
      for (int64_t jz = 0; jz < d->Jz; ++jz) {
        int64_t rz = rmod(T->kz[jz] * z, d->Nz);
        double czr = T->z.c[rz], czi = T->z.s[rz];
        double er = exyr * czr - exyi * czi, ei = exyr * czi + exyi * czr;
        const double* m = fh + 2 * (((jx * d->Jy + jy) * d->Jz + jz) * d->Jt);
        for (int64_t jt = 0; jt < d->Jt; ++jt) {
          int64_t rt = rmod(T->kt[jt] * t, d->Nt);
          double ctr = T->t.c[rt], cti = T->t.s[rt];
          double pr = er * ctr - ei * cti, pi = er * cti + ei * ctr;
          double wgt = scaled ? cweight(T->kt[jt], d->Nt) * invN : 1.0;
          accr += wgt * (m[2 * jt] * pr - m[2 * jt + 1] * pi);
        }
      }
    }
  }
  return accr;
}

static double gelu(double a) { return 0.5 * a * (1.0 + erf(a / sqrt(2.0))); }

static double gelu_grad(double a) {
  if (MUT(7)) return 0.5 * (1.0 + erf(a / sqrt(2.0)));
  return 0.5 * (1.0 + erf(a / sqrt(2.0))) + a * exp(-0.5 * a * a) / sqrt(TWO_PI);
}

/* values of the caller's inputs, FP32 or FP64 (dtype 0 / 1), promoted */
static inline double ld(const void* p, int dtype, int64_t i) {
  return dtype ? ((const double*)p)[i] : (double)((const float*)p)[i];
}

/* ======================================================================== */
/* exported entry points                                                     */
/* ======================================================================== */

int oracle_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

double oracle_gelu(double a) { return gelu(a); }
double oracle_gelu_grad(double a) { return gelu_grad(a); }

/* Kept-mode spectrum of nch real channels f[nch][Ng] -> fh[nch][Mk][2]. */
int oracle_spectrum(const int64_t* dims, int64_t nch, const double* f, double* fh,
                    int adjoint_scale) {
  dims_t d;
  if (dims_from(dims, &d) || !f || !fh || nch < 0) return ORC_EINVAL;
  tables_t T;
  work_t w;
  if (tables_make(&d, &T)) return ORC_ENOMEM;
  if (work_make(&d, &w)) { tables_free(&T); return ORC_ENOMEM; }
  for (int64_t c = 0; c < nch; ++c)
    spectrum_one(&d, &T, f + c * d.Ng, fh + 2 * c * d.Mk, adjoint_scale, &w);
  work_free(&w);
  tables_free(&T);
  return ORC_OK;
}

/* Real synthesis of nch kept spectra fh[nch][Mk][2] -> f[nch][Ng]. */
int oracle_synthesis(const int64_t* dims, int64_t nch, const double* fh, double* f, int scaled) {
  dims_t d;
  if (dims_from(dims, &d) || !f || !fh || nch < 0) return ORC_EINVAL;
  tables_t T;
  work_t w;
  if (tables_make(&d, &T)) return ORC_ENOMEM;
  if (work_make(&d, &w)) { tables_free(&T); return ORC_ENOMEM; }
  for (int64_t c = 0; c < nch; ++c)
    synthesis_one(&d, &T, fh + 2 * c * d.Mk, f + c * d.Ng, scaled, &w);
  work_free(&w);
  tables_free(&T);
  return ORC_OK;
}

/* The synthesis at npts points pts[npts][4] = (x,y,z,t): out[nch][npts]. */
int oracle_synthesis_points(const int64_t* dims, int64_t nch, const double* fh, int64_t npts,
                            const int64_t* pts, double* out, int scaled) {
  dims_t d;
  if (dims_from(dims, &d) || !fh || !pts || !out || nch < 0 || npts < 0) return ORC_EINVAL;
  tables_t T;
  if (tables_make(&d, &T)) return ORC_ENOMEM;
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t c = 0; c < nch; ++c)
    for (int64_t q = 0; q < npts; ++q)
      out[c * npts + q] = synthesis_point(&d, &T, fh + 2 * c * d.Mk, pts + 4 * q, scaled);
  tables_free(&T);
  return ORC_OK;
}

/* Literal 4-D sum of the spectrum: every term's phase from its own cos/sin. */
int oracle_spectrum_bruteforce(const int64_t* dims, int64_t nch, const double* f, double* fh,
                               int adjoint_scale) {
  dims_t d;
  if (dims_from(dims, &d) || !f || !fh || nch < 0) return ORC_EINVAL;
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t c = 0; c < nch; ++c) {
    for (int64_t m = 0; m < d.Mk; ++m) {
      int64_t jt = m % d.Jt, jz = (m / d.Jt) % d.Jz, jy = (m / (d.Jt * d.Jz)) % d.Jy,
              jx = m / (d.Jt * d.Jz * d.Jy);
      int64_t kx = kfreq(jx, d.mx), ky = kfreq(jy, d.my), kz = kfreq(jz, d.mz), kt = jt;
      double re = 0.0, im = 0.0;
      const double* src = f + c * d.Ng;
      for (int64_t p = 0; p < d.Ng; ++p) {
        int64_t t = p % d.Nt, z = (p / d.Nt) % d.Nz, y = (p / (d.Nt * d.Nz)) % d.Ny,
                x = p / (d.Nt * d.Nz * d.Ny);
        double ph = (double)rmod(kx * x, d.Nx) / (double)d.Nx + (double)rmod(ky * y, d.Ny) / (double)d.Ny +
                    (double)rmod(kz * z, d.Nz) / (double)d.Nz + (double)rmod(kt * t, d.Nt) / (double)d.Nt;
        double a = TWO_PI * ph;
        re += src[p] * cos(a);
        im -= src[p] * sin(a);
      }
      double s = adjoint_scale ? cweight(kt, d.Nt) / (double)d.Ng : 1.0;
      fh[2 * (c * d.Mk + m)] = re * s;
      fh[2 * (c * d.Mk + m) + 1] = im * s;
    }
  }
  return ORC_OK;
}

/* Literal 4-D synthesis sum. */
int oracle_synthesis_bruteforce(const int64_t* dims, int64_t nch, const double* fh, double* f,
                                int scaled) {
  dims_t d;
  if (dims_from(dims, &d) || !f || !fh || nch < 0) return ORC_EINVAL;
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t c = 0; c < nch; ++c) {
    for (int64_t p = 0; p < d.Ng; ++p) {
      int64_t t = p % d.Nt, z = (p / d.Nt) % d.Nz, y = (p / (d.Nt * d.Nz)) % d.Ny,
              x = p / (d.Nt * d.Nz * d.Ny);
      double acc = 0.0;
      for (int64_t m = 0; m < d.Mk; ++m) {
        int64_t jt = m % d.Jt, jz = (m / d.Jt) % d.Jz, jy = (m / (d.Jt * d.Jz)) % d.Jy,
                jx = m / (d.Jt * d.Jz * d.Jy);
        int64_t kx = kfreq(jx, d.mx), ky = kfreq(jy, d.my), kz = kfreq(jz, d.mz), kt = jt;
        double ph = (double)rmod(kx * x, d.Nx) / (double)d.Nx + (double)rmod(ky * y, d.Ny) / (double)d.Ny +
                    (double)rmod(kz * z, d.Nz) / (double)d.Nz + (double)rmod(kt * t, d.Nt) / (double)d.Nt;
        double a = TWO_PI * ph;
        double wgt = scaled ? cweight(kt, d.Nt) / (double)d.Ng : 1.0;
        const double* mm = fh + 2 * (c * d.Mk + m);
        acc += wgt * (mm[0] * cos(a) - mm[1] * sin(a));
      }
      f[c * d.Ng + p] = acc;
    }
  }
  return ORC_OK;
}

/* Spectral convolution, the einsum of Alg. 2: yh[b][o][j] = sum_i xh[b][i][j] w[i][o][j]. */
static void mix_forward(const dims_t* d, const double* xh, const void* w, int wtype, double* yh) {
  const int64_t Mk = d->Mk;
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t b = 0; b < d->B; ++b)
    for (int64_t o = 0; o < d->Co; ++o) {
      double* dst = yh + 2 * ((b * d->Co + o) * Mk);
      for (int64_t j = 0; j < Mk; ++j) { dst[2 * j] = 0.0; dst[2 * j + 1] = 0.0; }
      for (int64_t i = 0; i < d->Ci; ++i) {
        const double* a = xh + 2 * ((b * d->Ci + i) * Mk);
        int64_t wo = 2 * ((i * d->Co + o) * Mk);
        for (int64_t j = 0; j < Mk; ++j) {
          double ar = a[2 * j], ai = a[2 * j + 1];
          double wr = ld(w, wtype, wo + 2 * j), wi = ld(w, wtype, wo + 2 * j + 1);
          dst[2 * j] += ar * wr - ai * wi;
          dst[2 * j + 1] += ar * wi + ai * wr;
        }
      }
    }
}

/* dw[i][o][j] = sum_b conj(xh[b][i][j]) g[b][o][j];  gxh[b][i][j] = sum_o conj(w[i][o][j]) g[b][o][j] */
static void mix_adjoint(const dims_t* d, const double* xh, const void* w, int wtype,
                        const double* g, double* dw, double* gxh) {
  const int64_t Mk = d->Mk;
  if (dw) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t i = 0; i < d->Ci; ++i)
      for (int64_t o = 0; o < d->Co; ++o) {
        double* dst = dw + 2 * ((i * d->Co + o) * Mk);
        for (int64_t j = 0; j < Mk; ++j) { dst[2 * j] = 0.0; dst[2 * j + 1] = 0.0; }
        for (int64_t b = 0; b < d->B; ++b) {
          const double* a = xh + 2 * ((b * d->Ci + i) * Mk);
          const double* gg = g + 2 * ((b * d->Co + o) * Mk);
          for (int64_t j = 0; j < Mk; ++j) {
            double ar = a[2 * j], ai = (MUT(6) ? 1.0 : -1.0) * a[2 * j + 1];
            dst[2 * j] += ar * gg[2 * j] - ai * gg[2 * j + 1];
            dst[2 * j + 1] += ar * gg[2 * j + 1] + ai * gg[2 * j];
          }
        }
      }
  }
  if (gxh) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t b = 0; b < d->B; ++b)
      for (int64_t i = 0; i < d->Ci; ++i) {
        double* dst = gxh + 2 * ((b * d->Ci + i) * Mk);
        for (int64_t j = 0; j < Mk; ++j) { dst[2 * j] = 0.0; dst[2 * j + 1] = 0.0; }
        for (int64_t o = 0; o < d->Co; ++o) {
          int64_t wo = 2 * ((i * d->Co + o) * Mk);
          const double* gg = g + 2 * ((b * d->Co + o) * Mk);
          for (int64_t j = 0; j < Mk; ++j) {
            double wr = ld(w, wtype, wo + 2 * j), wi = -ld(w, wtype, wo + 2 * j + 1);
            dst[2 * j] += wr * gg[2 * j] - wi * gg[2 * j + 1];
            dst[2 * j + 1] += wr * gg[2 * j + 1] + wi * gg[2 * j];
          }
        }
      }
  }
}

int oracle_mix(const int64_t* dims, const double* xh, const double* w, double* yh) {
  dims_t d;
  if (dims_from(dims, &d) || !xh || !w || !yh) return ORC_EINVAL;
  mix_forward(&d, xh, w, 1, yh);
  return ORC_OK;
}

int oracle_mix_adjoint(const int64_t* dims, const double* xh, const double* w, const double* g,
                       double* dw, double* gxh) {
  dims_t d;
  if (dims_from(dims, &d) || !xh || !w || !g) return ORC_EINVAL;
  mix_adjoint(&d, xh, w, 1, g, dw, gxh);
  return ORC_OK;
}

/* Xh[b][i] of the caller's input x[B][Ci][Ng] (FP32 or FP64). */
static int input_spectrum(const dims_t* d, const tables_t* T, work_t* w, const void* x, int dtype,
                          double* xh, double* chan) {
  for (int64_t b = 0; b < d->B; ++b)
    for (int64_t i = 0; i < d->Ci; ++i) {
      int64_t off = (b * d->Ci + i) * d->Ng;
#pragma omp parallel for schedule(static)
      for (int64_t p = 0; p < d->Ng; ++p) chan[p] = ld(x, dtype, off + p);
      spectrum_one(d, T, chan, xh + 2 * ((b * d->Ci + i) * d->Mk), 0, w);
    }
  return ORC_OK;
}

/* A at one point of output channel o (spectral value s given). */
static double pre_activation(const dims_t* d, const void* x, const void* wl, const void* bias,
                             int dtype, int64_t b, int64_t o, int64_t p, double s) {
  double a = s + ld(bias, dtype, o);
  for (int64_t i = 0; i < d->Ci; ++i)
    a += ld(x, dtype, (b * d->Ci + i) * d->Ng + p) *
         ld(wl, dtype, MUT(5) ? o * d->Ci + i : i * d->Co + o);
  return a;
}

static int64_t point_index(const dims_t* d, const int64_t* p) {
  return ((p[0] * d->Ny + p[1]) * d->Nz + p[2]) * d->Nt + p[3];
}

/*
 * Block (with_linear = 1) or spectral convolution alone (with_linear = 0)
 * forward.  Inputs x[B][Ci][Ng], w[Ci][Co][Mk][2], wl[Ci][Co], bias[Co] are
 * FP32 (dtype 0) or FP64 (dtype 1); wl and bias are ignored without the
 * linear part.  Outputs (FP64, each nullable): z[B][Co][Ng] everywhere, and
 * z_pts[B][Co][npts] at the points pts[npts][4].
 */
int oracle_block_fwd(const int64_t* dims, int with_linear, int dtype, const void* x, const void* w,
                     const void* wl, const void* bias, double* z, int64_t npts, const int64_t* pts,
                     double* z_pts) {
  dims_t d;
  if (dims_from(dims, &d) || !x || !w) return ORC_EINVAL;
  if (with_linear && (!wl || !bias || d.Ci <= 0)) return ORC_EINVAL;
  if (npts > 0 && (!pts || !z_pts)) return ORC_EINVAL;
  for (int64_t q = 0; q < npts; ++q)
    if (pts[4 * q] < 0 || pts[4 * q] >= d.Nx || pts[4 * q + 1] < 0 || pts[4 * q + 1] >= d.Ny ||
        pts[4 * q + 2] < 0 || pts[4 * q + 2] >= d.Nz || pts[4 * q + 3] < 0 || pts[4 * q + 3] >= d.Nt)
      return ORC_EINVAL;
  tables_t T;
  work_t wk;
  if (tables_make(&d, &T)) return ORC_ENOMEM;
  if (work_make(&d, &wk)) { tables_free(&T); return ORC_ENOMEM; }
  double* xh = (double*)malloc(sizeof(double) * (size_t)(2 * d.B * d.Ci * d.Mk));
  double* yh = (double*)malloc(sizeof(double) * (size_t)(2 * d.B * d.Co * d.Mk));
  double* chan = (double*)malloc(sizeof(double) * (size_t)d.Ng);
  int rc = ORC_OK;
  if (!xh || !yh || !chan) { rc = ORC_ENOMEM; goto done; }
  input_spectrum(&d, &T, &wk, x, dtype, xh, chan);
  mix_forward(&d, xh, w, dtype, yh);
  for (int64_t b = 0; b < d.B; ++b)
    for (int64_t o = 0; o < d.Co; ++o) {
      const double* sp = yh + 2 * ((b * d.Co + o) * d.Mk);
      if (z) {
        double* dst = z + (b * d.Co + o) * d.Ng;
        synthesis_one(&d, &T, sp, dst, 1, &wk);
        if (with_linear) {
#pragma omp parallel for schedule(static)
          for (int64_t p = 0; p < d.Ng; ++p)
            dst[p] = gelu(pre_activation(&d, x, wl, bias, dtype, b, o, p, dst[p]));
        }
      }
      if (npts > 0) {
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < npts; ++q) {
          double s = synthesis_point(&d, &T, sp, pts + 4 * q, 1);
          if (with_linear)
            s = gelu(pre_activation(&d, x, wl, bias, dtype, b, o, point_index(&d, pts + 4 * q), s));
          z_pts[(b * d.Co + o) * npts + q] = s;
        }
      }
    }
done:
  free(xh); free(yh); free(chan);
  work_free(&wk);
  tables_free(&T);
  return rc;
}

/*
 * Gradient of the block (with_linear = 1) or of the spectral convolution alone
 * (with_linear = 0) for the upstream gradient dz[B][Co][Ng].  Outputs (FP64,
 * each nullable, overwritten): dx[B][Ci][Ng], dx_pts[B][Ci][npts] at pts,
 * dw[Ci][Co][Mk][2] = (dL/dRe W, dL/dIm W), dwl[Ci][Co], db[Co].
 */
int oracle_block_bwd(const int64_t* dims, int with_linear, int dtype, const void* x, const void* w,
                     const void* wl, const void* bias, const void* dz, double* dx, int64_t npts,
                     const int64_t* pts, double* dx_pts, double* dw, double* dwl, double* db) {
  dims_t d;
  if (dims_from(dims, &d) || !x || !w || !dz) return ORC_EINVAL;
  if (with_linear && (!wl || !bias)) return ORC_EINVAL;
  if (npts > 0 && (!pts || !dx_pts)) return ORC_EINVAL;
  for (int64_t q = 0; q < npts; ++q)
    if (pts[4 * q] < 0 || pts[4 * q] >= d.Nx || pts[4 * q + 1] < 0 || pts[4 * q + 1] >= d.Ny ||
        pts[4 * q + 2] < 0 || pts[4 * q + 2] >= d.Nz || pts[4 * q + 3] < 0 || pts[4 * q + 3] >= d.Nt)
      return ORC_EINVAL;
  tables_t T;
  work_t wk;
  if (tables_make(&d, &T)) return ORC_ENOMEM;
  if (work_make(&d, &wk)) { tables_free(&T); return ORC_ENOMEM; }
  const int64_t Ng = d.Ng, Mk = d.Mk;
  double* xh = (double*)malloc(sizeof(double) * (size_t)(2 * d.B * d.Ci * Mk));
  double* yh = (double*)malloc(sizeof(double) * (size_t)(2 * d.B * d.Co * Mk));
  double* g = (double*)malloc(sizeof(double) * (size_t)(2 * d.B * d.Co * Mk));
  double* gxh = (double*)malloc(sizeof(double) * (size_t)(2 * d.B * d.Ci * Mk));
  double* da = (double*)malloc(sizeof(double) * (size_t)Ng);
  double* chan = (double*)malloc(sizeof(double) * (size_t)Ng);
  double* da_pts = npts > 0 ? (double*)malloc(sizeof(double) * (size_t)(d.B * d.Co * npts)) : NULL;
  int rc = ORC_OK;
  if (!xh || !yh || !g || !gxh || !da || !chan || (npts > 0 && !da_pts)) {
    rc = ORC_ENOMEM;
    goto done;
  }
  if (dx) memset(dx, 0, sizeof(double) * (size_t)(d.B * d.Ci * Ng));
  if (dwl) memset(dwl, 0, sizeof(double) * (size_t)(d.Ci * d.Co));
  if (db) memset(db, 0, sizeof(double) * (size_t)d.Co);

  input_spectrum(&d, &T, &wk, x, dtype, xh, chan);
  if (with_linear) mix_forward(&d, xh, w, dtype, yh);

  for (int64_t b = 0; b < d.B; ++b)
    for (int64_t o = 0; o < d.Co; ++o) {
      const int64_t zoff = (b * d.Co + o) * Ng;
      if (with_linear) {
        /* recompute A on the whole grid, then dA = dZ GELU'(A) */
        synthesis_one(&d, &T, yh + 2 * ((b * d.Co + o) * Mk), da, 1, &wk);
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < Ng; ++p) {
          double a = pre_activation(&d, x, wl, bias, dtype, b, o, p, da[p]);
          da[p] = ld(dz, dtype, zoff + p) * gelu_grad(a);
        }
        double sdb = 0.0;
#pragma omp parallel for reduction(+ : sdb) schedule(static)
        for (int64_t p = 0; p < Ng; ++p) sdb += da[p];
        if (db) db[o] += sdb;
        if (dwl) {
          for (int64_t i = 0; i < d.Ci; ++i) {
            double s = 0.0;
            const int64_t xoff = (b * d.Ci + i) * Ng;
#pragma omp parallel for reduction(+ : s) schedule(static)
            for (int64_t p = 0; p < Ng; ++p) s += ld(x, dtype, xoff + p) * da[p];
            dwl[i * d.Co + o] += s;
          }
        }
        if (dx) {
          for (int64_t i = 0; i < d.Ci; ++i) {
            double wio = ld(wl, dtype, i * d.Co + o);
            double* dst = dx + (b * d.Ci + i) * Ng;
#pragma omp parallel for schedule(static)
            for (int64_t p = 0; p < Ng; ++p) dst[p] += wio * da[p];
          }
        }
      } else {
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < Ng; ++p) da[p] = ld(dz, dtype, zoff + p);
      }
      for (int64_t q = 0; q < npts; ++q) da_pts[(b * d.Co + o) * npts + q] = da[point_index(&d, pts + 4 * q)];
      spectrum_one(&d, &T, da, g + 2 * ((b * d.Co + o) * Mk), 1, &wk);
    }

  mix_adjoint(&d, xh, w, dtype, g, dw, gxh);

  for (int64_t b = 0; b < d.B; ++b)
    for (int64_t i = 0; i < d.Ci; ++i) {
      const double* sp = gxh + 2 * ((b * d.Ci + i) * Mk);
      if (dx) {
        double* dst = dx + (b * d.Ci + i) * Ng;
        synthesis_one(&d, &T, sp, chan, 0, &wk);
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < Ng; ++p) dst[p] += chan[p];
      }
      if (npts > 0) {
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < npts; ++q) {
          double s = synthesis_point(&d, &T, sp, pts + 4 * q, 0);
          if (with_linear)
            for (int64_t o = 0; o < d.Co; ++o)
              s += ld(wl, dtype, i * d.Co + o) * da_pts[(b * d.Co + o) * npts + q];
          dx_pts[(b * d.Ci + i) * npts + q] = s;
        }
      }
    }
done:
  free(xh); free(yh); free(g); free(gxh); free(da); free(chan); free(da_pts);
  work_free(&wk);
  tables_free(&T);
  return rc;
}

/* ======================================================================== */
/* The layers around the blocks (Alg. 1): encoder and decoder 1x1 layers,    */
/* and the training loss                                                     */
/* ======================================================================== */
/*
 * Pointwise channel layer (Alg. 1's encoder X W^e and decoder X W^d, each
 * followed by sigma; the bias of the original FNO's 1x1 layers is optional):
 *   A[b,o,p] = sum_i X[b,i,p] W[i,o] + bias[o]      W stored [Ci][Co]
 *   Y        = sigma(A),  sigma = identity (act 0) or GELU (act 1)
 * Gradient for an upstream dY:
 *   dA = dY sigma'(A);  dX[b,i,p] = sum_o W[i,o] dA[b,o,p]
 *   dW[i,o] = sum_{b,p} X[b,i,p] dA[b,o,p];  db[o] = sum_{b,p} dA[b,o,p]
 * Loss (mean squared error against a target T over n values):
 *   L = (1/n) sum (Y - T)^2;  dY = (2/n) (Y - T)
 */
static double pw_pre(int64_t Ci, int64_t Co, int64_t P, int dtype, const void* x, const void* w,
                     const void* bias, int64_t b, int64_t o, int64_t p) {
  double a = (bias && !MUT(8)) ? ld(bias, dtype, o) : 0.0;
  for (int64_t i = 0; i < Ci; ++i) a += ld(x, dtype, (b * Ci + i) * P + p) * ld(w, dtype, i * Co + o);
  return a;
}

int oracle_pointwise_fwd(int64_t B, int64_t Ci, int64_t Co, int64_t P, int act, int dtype,
                         const void* x, const void* w, const void* bias, double* y) {
  if (B < 0 || Ci < 1 || Co < 1 || P < 0 || (act != 0 && act != 1) || !w || !y) return ORC_EINVAL;
  if (B * P > 0 && !x) return ORC_EINVAL;
  for (int64_t b = 0; b < B; ++b)
    for (int64_t o = 0; o < Co; ++o) {
#pragma omp parallel for schedule(static)
      for (int64_t p = 0; p < P; ++p) {
        const double a = pw_pre(Ci, Co, P, dtype, x, w, bias, b, o, p);
        y[(b * Co + o) * P + p] = act ? gelu(a) : a;
      }
    }
  return ORC_OK;
}

int oracle_pointwise_bwd(int64_t B, int64_t Ci, int64_t Co, int64_t P, int act, int dtype,
                         const void* x, const void* w, const void* bias, const void* dy,
                         double* dx, double* dw, double* db) {
  if (B < 0 || Ci < 1 || Co < 1 || P < 0 || (act != 0 && act != 1) || !w || !dw) return ORC_EINVAL;
  if (B * P > 0 && (!x || !dy)) return ORC_EINVAL;
  double* da = (double*)malloc(sizeof(double) * (size_t)(B * Co * P > 0 ? B * Co * P : 1));
  if (!da) return ORC_ENOMEM;
  for (int64_t b = 0; b < B; ++b)
    for (int64_t o = 0; o < Co; ++o) {
#pragma omp parallel for schedule(static)
      for (int64_t p = 0; p < P; ++p) {
        const int64_t e = (b * Co + o) * P + p;
        double s = 1.0;
        if (act) {
          const double a = pw_pre(Ci, Co, P, dtype, x, w, bias, b, o, p);
          s = gelu_grad(MUT(10) ? gelu(a) : a);
        }
        da[e] = ld(dy, dtype, e) * s;
      }
    }
  for (int64_t i = 0; i < Ci; ++i)
    for (int64_t o = 0; o < Co; ++o) {
      double acc = 0.0;
      for (int64_t b = 0; b < B; ++b) {
#pragma omp parallel for schedule(static) reduction(+ : acc)
        for (int64_t p = 0; p < P; ++p)
          acc += ld(x, dtype, (b * Ci + i) * P + p) * da[(b * Co + o) * P + p];
      }
      dw[i * Co + o] = acc;
    }
  if (db)
    for (int64_t o = 0; o < Co; ++o) {
      double acc = 0.0;
      for (int64_t b = 0; b < B; ++b) {
#pragma omp parallel for schedule(static) reduction(+ : acc)
        for (int64_t p = 0; p < P; ++p) acc += da[(b * Co + o) * P + p];
      }
      db[o] = acc;
    }
  if (dx)
    for (int64_t b = 0; b < B; ++b)
      for (int64_t i = 0; i < Ci; ++i) {
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < P; ++p) {
          double s = 0.0;
          for (int64_t o = 0; o < Co; ++o) s += ld(w, dtype, i * Co + o) * da[(b * Co + o) * P + p];
          dx[(b * Ci + i) * P + p] = s;
        }
      }
  free(da);
  return ORC_OK;
}

int oracle_mse(int64_t n, int dtype, const void* y, const void* t, double* loss, double* dy) {
  if (n < 1 || !y || !t || !loss) return ORC_EINVAL;
  double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
  for (int64_t e = 0; e < n; ++e) {
    const double r = ld(y, dtype, e) - ld(t, dtype, e);
    acc += r * r;
    if (dy) dy[e] = (MUT(9) ? 1.0 : 2.0) * r / (double)n;
  }
  *loss = acc / (double)n;
  return ORC_OK;
}

/* ======================================================================== */
/* Training step: Adam (Kingma and Ba), the optimizer of the original FNO     */
/* ======================================================================== */
/*
 * For step t >= 1 with gradient g:
 *   m = b1 m + (1 - b1) g;   v = b2 v + (1 - b2) g^2
 *   p = p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
 * p, m, v updated in place (FP64); g read as FP32 or FP64 (dtype 0 / 1).
 */
int oracle_adam(int64_t n, int dtype, double* p, const void* g, double* m, double* v, double lr,
                double b1, double b2, double eps, int64_t t) {
  if (n < 0 || t < 1 || !(b1 >= 0.0 && b1 < 1.0) || !(b2 >= 0.0 && b2 < 1.0) || !(eps > 0.0))
    return ORC_EINVAL;
  if (n > 0 && (!p || !g || !m || !v)) return ORC_EINVAL;
  const double bc1 = 1.0 - pow(b1, (double)t), bc2 = 1.0 - pow(b2, (double)t);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < n; ++e) {
    const double gr = ld(g, dtype, e);
    m[e] = b1 * m[e] + (1.0 - b1) * gr;
    v[e] = b2 * v[e] + (1.0 - b2) * gr * (MUT(11) ? 1.0 : gr);
    p[e] -= lr * (m[e] / bc1) / (sqrt(v[e] / bc2) + eps);
  }
  return ORC_OK;
}
