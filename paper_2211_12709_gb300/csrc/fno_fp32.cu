// fno_fp32.cu -- the FP32 CUDA-core form of every stage of the spectral FNO
// block (the "plain form"), plus the table, reduction and fill kernels that
// every precision shares.
//
// Stage map (Alg. 2, Sec. IV-C of the paper; the forward truncated DFT runs
// over the non-partitioned axes y, z, t first and over x last, the inverse is
// the same chain in reverse order):
//   k_fwd_tz_f32   pruned DFT over t then z of each (b, c, x, y) column
//   k_line_f32     one complex DFT axis (forward y, x; inverse x, y)
//   k_mix_f32      per-mode complex channel mixing (the einsum of Alg. 2)
//   k_mix_adj_f32  its adjoint: weight gradient and input-spectrum gradient
//   k_epi_f32      inverse z then t, fused with the 1x1 linear, bias and GELU
//                  (or their gradients)
#include <algorithm>

#include "fno_internal.h"

namespace fno {

#define FNO_LAUNCH(name, kern, grid, block, smem, stream, ...)   \
  do {                                                           \
    prof_before(name, stream);                                   \
    kern<<<grid, block, smem, stream>>>(__VA_ARGS__);            \
    cudaError_t e_ = cudaGetLastError();                         \
    prof_after(stream);                                          \
    if (e_ != cudaSuccess) return e_;                            \
  } while (0)

static int persistent_grid(const void* kern, int threads, size_t smem, int64_t work) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  int64_t g = (int64_t)per_sm * sm_count();
  if (g > work) g = work;
  if (g < 1) g = 1;
  return (int)g;
}

static cudaError_t allow_smem(const void* kern, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// ---------------------------------------------------------------------------
// Basis tables: exp(sign * 2 pi i * (k n mod N) / N), evaluated in FP64 with
// sincospi on the exactly reduced residue, optionally scaled by c(kt)/Ng.
// ---------------------------------------------------------------------------
struct TabSeg {
  float2* dst;
  int rows, cols, N, m, k_on_row, sign, scale;
};
struct TabParams {
  TabSeg seg[10];
  long long start[11];
  int nseg;
  int Nt;
  double invNg;
  int* err;
};

__global__ void k_tables(TabParams p) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx == 0 && p.err) *p.err = 0;
  if (idx >= p.start[p.nseg]) return;
  int s = 0;
  while (s + 1 < p.nseg && idx >= p.start[s + 1]) ++s;
  const TabSeg g = p.seg[s];
  long long e = idx - p.start[s];
  int r = (int)(e / g.cols), c = (int)(e % g.cols);
  int j = g.k_on_row ? r : c;
  int n = g.k_on_row ? c : r;
  long long k = (g.m > 0) ? (j < g.m ? j : j - 2 * g.m) : j;
  long long rr = (k * n) % g.N;
  if (rr < 0) rr += g.N;
  double sn, cs;
  sincospi(2.0 * (double)rr / (double)g.N, &sn, &cs);
  double sc = 1.0;
  if (g.scale) {
    bool single = (k == 0) || ((p.Nt % 2 == 0) && (2 * k == p.Nt));
    sc = (single ? 1.0 : 2.0) * p.invNg;
  }
  g.dst[e] = make_float2((float)(cs * sc), (float)((double)g.sign * sn * sc));
}

cudaError_t launch_tables(const Dims& d, const Tables& T, int* err, cudaStream_t s) {
  TabParams p{};
  p.err = err;
  auto add = [&](float2* dst, int64_t rows, int64_t cols, int64_t N, int64_t m, int kr, int sign,
                 int scale) {
    p.seg[p.nseg] = TabSeg{dst, (int)rows, (int)cols, (int)N, (int)m, kr, sign, scale};
    p.start[p.nseg + 1] = p.start[p.nseg] + rows * cols;
    ++p.nseg;
  };
  p.start[0] = 0;
  add(T.Fx, d.Jx, d.Nx, d.Nx, d.mx, 1, -1, 0);
  add(T.Fy, d.Jy, d.Ny, d.Ny, d.my, 1, -1, 0);
  add(T.Fz, d.Jz, d.Nz, d.Nz, d.mz, 1, -1, 0);
  add(T.Ft, d.Jt, d.Nt, d.Nt, 0, 1, -1, 0);
  add(T.Fta, d.Jt, d.Nt, d.Nt, 0, 1, -1, 1);
  add(T.Ix, d.Nx, d.Jx, d.Nx, d.mx, 0, +1, 0);
  add(T.Iy, d.Ny, d.Jy, d.Ny, d.my, 0, +1, 0);
  add(T.Iz, d.Nz, d.Jz, d.Nz, d.mz, 0, +1, 0);
  add(T.Its, d.Jt, d.Nt, d.Nt, 0, 1, +1, 1);
  add(T.Itu, d.Jt, d.Nt, d.Nt, 0, 1, +1, 0);
  p.Nt = (int)d.Nt;
  p.invNg = 1.0 / (double)d.Ng;
  long long total = p.start[p.nseg];
  int threads = 256;
  int blocks = (int)((total + threads - 1) / threads);
  FNO_LAUNCH("fno_tables", k_tables, blocks, threads, 0, s, p);
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Forward pruned DFT over t, then z, of each column [Nz][Nt] (real input):
//   P[z][jt]  = sum_t x[z][t] ft[jt][t]
//   T1[jz][jt] = sum_z fz[jz][z] P[z][jt]
// One CTA walks columns (persistent); one thread per z row in the t stage and
// per (jz, jt) output in the z stage.
// ---------------------------------------------------------------------------
size_t fwd_tz_smem_bytes(const Dims& d) {
  return sizeof(float2) * (size_t)(d.Jt * d.Nt + d.Jz * (d.Nz + 1) + d.Nz * d.Jt);
}

template <bool VEC4>
__global__ void __launch_bounds__(128)
    k_fwd_tz_f32(const float* __restrict__ in, float2* __restrict__ out, long long ncol, int Nz,
                 int Nt, int Jz, int Jt, const float2* __restrict__ ft,
                 const float2* __restrict__ fz) {
  extern __shared__ float4 smem4[];
  float2* sFt = reinterpret_cast<float2*>(smem4);  // [Jt][Nt]
  float2* sFz = sFt + Jt * Nt;                      // [Jz][Nz + 1]
  float2* sP = sFz + Jz * (Nz + 1);                 // [Nz][Jt]
  for (int e = threadIdx.x; e < Jt * Nt; e += blockDim.x) sFt[e] = ft[e];
  for (int e = threadIdx.x; e < Jz * Nz; e += blockDim.x) {
    int r = e / Nz, c = e - r * Nz;
    sFz[r * (Nz + 1) + c] = fz[e];
  }
  __syncthreads();
  const int JZT = Jz * Jt;
  for (long long col = blockIdx.x; col < ncol; col += gridDim.x) {
    const float* src = in + col * (long long)Nz * Nt;
    for (int z = threadIdx.x; z < Nz; z += blockDim.x) {
      const float* row = src + (long long)z * Nt;
      for (int j0 = 0; j0 < Jt; j0 += 8) {
        float ar[8], ai[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) { ar[q] = 0.f; ai[q] = 0.f; }
        if (VEC4) {
          for (int t = 0; t < Nt; t += 4) {
            float4 v4 = __ldg(reinterpret_cast<const float4*>(row + t));
            float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                if (j0 + q < Jt) {
                  float2 f = sFt[(j0 + q) * Nt + t + u];
                  ar[q] = fmaf(vv[u], f.x, ar[q]);
                  ai[q] = fmaf(vv[u], f.y, ai[q]);
                }
              }
            }
          }
        } else {
          for (int t = 0; t < Nt; ++t) {
            float v = __ldg(row + t);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              if (j0 + q < Jt) {
                float2 f = sFt[(j0 + q) * Nt + t];
                ar[q] = fmaf(v, f.x, ar[q]);
                ai[q] = fmaf(v, f.y, ai[q]);
              }
            }
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (j0 + q < Jt) sP[z * Jt + j0 + q] = make_float2(ar[q], ai[q]);
      }
    }
    __syncthreads();
    float2* dst = out + col * (long long)JZT;
    for (int o = threadIdx.x; o < JZT; o += blockDim.x) {
      int jz = o / Jt, jt = o - jz * Jt;
      const float2* f = sFz + jz * (Nz + 1);
      float re = 0.f, im = 0.f;
      for (int z = 0; z < Nz; ++z) {
        float2 a = f[z], b = sP[z * Jt + jt];
        re = fmaf(a.x, b.x, re);
        re = fmaf(-a.y, b.y, re);
        im = fmaf(a.x, b.y, im);
        im = fmaf(a.y, b.x, im);
      }
      dst[o] = make_float2(re, im);
    }
    __syncthreads();
  }
}

cudaError_t launch_fwd_tz_f32(const float* in, float2* out, int64_t ncol, const Dims& d,
                              const float2* ft, const float2* fz, cudaStream_t s) {
  if (ncol <= 0) return cudaSuccess;
  size_t smem = fwd_tz_smem_bytes(d);
  const int threads = 128;
  if (d.Nt % 4 == 0) {
    const void* k = (const void*)k_fwd_tz_f32<true>;
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    int grid = persistent_grid(k, threads, smem, ncol);
    FNO_LAUNCH("fno_fwd_tz_f32", k_fwd_tz_f32<true>, grid, threads, smem, s, in, out,
               (long long)ncol, (int)d.Nz, (int)d.Nt, (int)d.Jz, (int)d.Jt, ft, fz);
  } else {
    const void* k = (const void*)k_fwd_tz_f32<false>;
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    int grid = persistent_grid(k, threads, smem, ncol);
    FNO_LAUNCH("fno_fwd_tz_f32", k_fwd_tz_f32<false>, grid, threads, smem, s, in, out,
               (long long)ncol, (int)d.Nz, (int)d.Nt, (int)d.Jz, (int)d.Jt, ft, fz);
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// One complex DFT axis: out[o][q][i] = sum_n tab[q][n] in[o][n][i].
// A CTA stages an [nin][32] slab of the input in shared memory; a warp owns a
// group of QB output rows for 32 consecutive i.
// ---------------------------------------------------------------------------
size_t line_smem_bytes(int nin, int nout) {
  return sizeof(float2) * (size_t)(nout * nin + nin * 32);
}

template <int QB>
__global__ void __launch_bounds__(256)
    k_line_f32(const float2* __restrict__ in, float2* __restrict__ out, long long outer, int nin,
               int nout, long long inner, const float2* __restrict__ tab) {
  extern __shared__ float4 smem4[];
  float2* sTab = reinterpret_cast<float2*>(smem4);  // [nout][nin]
  float2* sIn = sTab + nout * nin;                   // [nin][32]
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + lane;
  for (int e = tid; e < nout * nin; e += 256) sTab[e] = tab[e];
  const long long ntile = (inner + 31) / 32;
  const long long nwork = outer * ntile;
  for (long long w = blockIdx.x; w < nwork; w += gridDim.x) {
    const long long o = w / ntile;
    const long long i = (w - o * ntile) * 32 + lane;
    const bool ok = i < inner;
    __syncthreads();
    for (int n = ty; n < nin; n += 8)
      sIn[n * 32 + lane] = ok ? in[(o * nin + n) * inner + i] : make_float2(0.f, 0.f);
    __syncthreads();
    for (int q0 = ty * QB; q0 < nout; q0 += 8 * QB) {
      float2 acc[QB];
#pragma unroll
      for (int qq = 0; qq < QB; ++qq) acc[qq] = make_float2(0.f, 0.f);
      for (int n = 0; n < nin; ++n) {
        float2 v = sIn[n * 32 + lane];
#pragma unroll
        for (int qq = 0; qq < QB; ++qq) {
          if (q0 + qq < nout) {
            float2 f = sTab[(q0 + qq) * nin + n];
            acc[qq].x = fmaf(f.x, v.x, acc[qq].x);
            acc[qq].x = fmaf(-f.y, v.y, acc[qq].x);
            acc[qq].y = fmaf(f.x, v.y, acc[qq].y);
            acc[qq].y = fmaf(f.y, v.x, acc[qq].y);
          }
        }
      }
      if (ok) {
#pragma unroll
        for (int qq = 0; qq < QB; ++qq)
          if (q0 + qq < nout) out[(o * nout + q0 + qq) * inner + i] = acc[qq];
      }
    }
  }
}

cudaError_t launch_line_f32(const float2* in, float2* out, int64_t outer, int nin, int nout,
                            int64_t inner, const float2* tab, cudaStream_t s) {
  if (outer <= 0 || inner <= 0) return cudaSuccess;
  size_t smem = line_smem_bytes(nin, nout);
  const void* k = (const void*)k_line_f32<4>;
  cudaError_t e = allow_smem(k, smem);
  if (e != cudaSuccess) return e;
  int64_t work = outer * ((inner + 31) / 32);
  int grid = persistent_grid(k, 256, smem, work);
  FNO_LAUNCH("fno_line_f32", k_line_f32<4>, grid, dim3(32, 8), smem, s, in, out,
             (long long)outer, nin, nout, (long long)inner, tab);
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Spectral convolution and its adjoint (FP32).  One thread per mode j; the
// batch is held in registers in chunks of BC.
// ---------------------------------------------------------------------------
template <int BC>
__global__ void __launch_bounds__(128)
    k_mix_f32(const float2* __restrict__ xh, const float2* __restrict__ w, float2* __restrict__ yh,
              int B, int Ci, int Co, long long Mk) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int o = blockIdx.y;
  if (j >= Mk) return;
  for (int b0 = 0; b0 < B; b0 += BC) {
    float2 acc[BC];
#pragma unroll
    for (int q = 0; q < BC; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int i = 0; i < Ci; ++i) {
      const float2 wv = w[((long long)i * Co + o) * Mk + j];
#pragma unroll
      for (int q = 0; q < BC; ++q) {
        if (b0 + q < B) {
          const float2 xv = xh[((long long)(b0 + q) * Ci + i) * Mk + j];
          acc[q].x = fmaf(xv.x, wv.x, acc[q].x);
          acc[q].x = fmaf(-xv.y, wv.y, acc[q].x);
          acc[q].y = fmaf(xv.x, wv.y, acc[q].y);
          acc[q].y = fmaf(xv.y, wv.x, acc[q].y);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < BC; ++q)
      if (b0 + q < B) yh[((long long)(b0 + q) * Co + o) * Mk + j] = acc[q];
  }
}

template <int BC>
__global__ void __launch_bounds__(128)
    k_mix_adj_f32(const float2* __restrict__ xh, const float2* __restrict__ w,
                  const float2* __restrict__ g, float2* __restrict__ dw, float2* __restrict__ gxh,
                  int B, int Ci, int Co, long long Mk) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= Mk) return;
  for (int b0 = 0; b0 < B; b0 += BC) {
    float2 xv[BC], ga[BC];
#pragma unroll
    for (int q = 0; q < BC; ++q) {
      xv[q] = (b0 + q < B) ? xh[((long long)(b0 + q) * Ci + i) * Mk + j] : make_float2(0.f, 0.f);
      ga[q] = make_float2(0.f, 0.f);
    }
    for (int o = 0; o < Co; ++o) {
      const long long widx = ((long long)i * Co + o) * Mk + j;
      const float2 wv = w[widx];
      float2 da = make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < BC; ++q) {
        if (b0 + q < B) {
          const float2 gv = g[((long long)(b0 + q) * Co + o) * Mk + j];
          // ga += conj(w) g
          ga[q].x = fmaf(wv.x, gv.x, ga[q].x);
          ga[q].x = fmaf(wv.y, gv.y, ga[q].x);
          ga[q].y = fmaf(wv.x, gv.y, ga[q].y);
          ga[q].y = fmaf(-wv.y, gv.x, ga[q].y);
          // da += conj(xh) g
          da.x = fmaf(xv[q].x, gv.x, da.x);
          da.x = fmaf(xv[q].y, gv.y, da.x);
          da.y = fmaf(xv[q].x, gv.y, da.y);
          da.y = fmaf(-xv[q].y, gv.x, da.y);
        }
      }
      if (dw) {
        if (b0 == 0) {
          dw[widx] = da;
        } else {
          float2 p = dw[widx];
          dw[widx] = make_float2(p.x + da.x, p.y + da.y);
        }
      }
    }
    if (gxh) {
#pragma unroll
      for (int q = 0; q < BC; ++q)
        if (b0 + q < B) gxh[((long long)(b0 + q) * Ci + i) * Mk + j] = ga[q];
    }
  }
}

cudaError_t launch_mix_f32(const Dims& d, const float2* xh, const float2* w, float2* yh,
                           cudaStream_t s) {
  if (d.B <= 0) return cudaSuccess;
  dim3 grid((unsigned)((d.Mk + 127) / 128), (unsigned)d.Co);
  FNO_LAUNCH("fno_mix_f32", k_mix_f32<4>, grid, 128, 0, s, xh, w, yh, (int)d.B, (int)d.Ci,
             (int)d.Co, (long long)d.Mk);
  return cudaSuccess;
}

cudaError_t launch_mix_adjoint_f32(const Dims& d, const float2* xh, const float2* w,
                                   const float2* g, float2* dw, float2* gxh, cudaStream_t s) {
  if (d.B <= 0) return cudaSuccess;
  dim3 grid((unsigned)((d.Mk + 127) / 128), (unsigned)d.Ci);
  FNO_LAUNCH("fno_mix_adjoint_f32", k_mix_adj_f32<4>, grid, 128, 0, s, xh, w, g, dw, gxh,
             (int)d.B, (int)d.Ci, (int)d.Co, (long long)d.Mk);
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Inverse z, t stages fused with the pointwise epilogue.
// A CTA owns one (b, x, y) column at a time and all its channels.  For each
// chunk of zc z-planes:
//   phase 1  Q[c][z][jt] = sum_jz Iz[z][jz] U[c][jz][jt]
//   phase 2  one thread per point (z, t):
//            S_c = sum_jt Re(Q[c][z][jt] It[jt][t]),  lin_c = sum_i Wl(i, c) L_i
//            SPECTRAL: out = S      FWD: out = GELU(S + lin + bias)
//            DA: out = dz GELU'(S + lin + bias)      DX: out = S + lin
//   phase 3  (DA) per-CTA sums of x_i dA_c and dA_c, Kahan-compensated
// ---------------------------------------------------------------------------
struct EpiK {
  EpiArgs a;
  long long B, Nx, Ny;
  int Nz, Nt, Jz, Jt, zc;
};

static int epi_zc(const Dims& d) {
  int zc = (int)std::max<int64_t>(1, 256 / d.Nt);
  if (zc > d.Nz) zc = (int)d.Nz;
  return zc;
}

size_t epilogue_smem_bytes(const Dims& d, int mode, int Cs, int Cl) {
  const int zc = epi_zc(d);
  const size_t PP = (size_t)zc * d.Nt + 1;
  size_t b = sizeof(float2) * (size_t)(Cs * d.Jz * d.Jt + Cs * zc * d.Jt + d.Nz * (d.Jz + 1) +
                                       d.Jt * d.Nt);
  b += sizeof(float) * (size_t)(Cl * Cs + Cs);
  if (mode == EPI_DA) b += sizeof(float) * ((size_t)(Cl + Cs) * PP + 2 * (size_t)(Cl * Cs + Cs));
  return b;
}

int epilogue_max_grid() { return 1024; }

template <int MODE, int CLM>
__global__ void __launch_bounds__(256, 2) k_epi_f32(EpiK k) {
  extern __shared__ float4 smem4[];
  const EpiArgs& a = k.a;
  const int Cs = a.Cs, Cl = a.Cl, Jz = k.Jz, Jt = k.Jt, Nz = k.Nz, Nt = k.Nt, zc = k.zc;
  const int PP = zc * Nt + 1;
  float2* sU = reinterpret_cast<float2*>(smem4);  // [Cs][Jz][Jt]
  float2* sQ = sU + Cs * Jz * Jt;                  // [Cs][zc][Jt]
  float2* sIz = sQ + Cs * zc * Jt;                 // [Nz][Jz + 1]
  float2* sIt = sIz + Nz * (Jz + 1);               // [Jt][Nt]
  float* sW = reinterpret_cast<float*>(sIt + Jt * Nt);  // [Cl][Cs]
  float* sB = sW + Cl * Cs;                              // [Cs]
  float* sX = sB + Cs;                                   // DA: [Cl][PP]
  float* sD = sX + (MODE == EPI_DA ? Cl * PP : 0);       // DA: [Cs][PP]
  float* sAcc = sD + (MODE == EPI_DA ? Cs * PP : 0);     // DA: sums, then compensations
  const int npair = Cl * Cs + Cs;
  const int tid = threadIdx.x, nthr = blockDim.x;

  for (int e = tid; e < Nz * Jz; e += nthr) {
    int r = e / Jz, c = e - r * Jz;
    sIz[r * (Jz + 1) + c] = a.Iz[e];
  }
  for (int e = tid; e < Jt * Nt; e += nthr) sIt[e] = a.It[e];
  if (MODE != EPI_SPECTRAL) {
    for (int e = tid; e < Cl * Cs; e += nthr) {
      int i = e / Cs, c = e - i * Cs;
      sW[e] = a.wlin[(long long)i * a.w_si + (long long)c * a.w_sc];
    }
    for (int c = tid; c < Cs; c += nthr) sB[c] = (MODE == EPI_FWD || MODE == EPI_DA) ? a.bias[c] : 0.f;
  }
  if (MODE == EPI_DA)
    for (int e = tid; e < 2 * npair; e += nthr) sAcc[e] = 0.f;

  const long long NxNy = k.Nx * k.Ny;
  const long long plane = (long long)Nz * Nt;
  const long long chan = NxNy * plane;
  const long long ncol = k.B * NxNy;
  const int JZT = Jz * Jt;
  for (long long col = blockIdx.x; col < ncol; col += gridDim.x) {
    const long long b = col / NxNy;
    const long long xy = col - b * NxNy;
    __syncthreads();
    for (int e = tid; e < Cs * JZT; e += nthr) {
      int c = e / JZT, r = e - c * JZT;
      sU[e] = a.U[((b * Cs + c) * NxNy + xy) * JZT + r];
    }
    __syncthreads();
    for (int z0 = 0; z0 < Nz; z0 += zc) {
      const int zn = min(zc, Nz - z0);
      for (int e = tid; e < Cs * zn * Jt; e += nthr) {
        int jt = e % Jt;
        int zz = (e / Jt) % zn;
        int c = e / (Jt * zn);
        const float2* iz = sIz + (z0 + zz) * (Jz + 1);
        const float2* u = sU + c * JZT + jt;
        float re = 0.f, im = 0.f;
        for (int jz = 0; jz < Jz; ++jz) {
          float2 f = iz[jz], v = u[jz * Jt];
          re = fmaf(f.x, v.x, re);
          re = fmaf(-f.y, v.y, re);
          im = fmaf(f.x, v.y, im);
          im = fmaf(f.y, v.x, im);
        }
        sQ[(c * zc + zz) * Jt + jt] = make_float2(re, im);
      }
      __syncthreads();
      for (int pt = tid; pt < zn * Nt; pt += nthr) {
        const int zz = pt / Nt, t = pt - zz * Nt;
        const long long pofs = xy * plane + (long long)(z0 + zz) * Nt + t;
        float L[CLM];
        if (MODE != EPI_SPECTRAL) {
#pragma unroll
          for (int i = 0; i < CLM; ++i)
            L[i] = (i < Cl) ? a.lin_in[(b * Cl + i) * chan + pofs] : 0.f;
        }
        for (int c = 0; c < Cs; ++c) {
          const float2* q = sQ + (c * zc + zz) * Jt;
          float sv = 0.f;
          for (int jt = 0; jt < Jt; ++jt) {
            float2 qv = q[jt], iv = sIt[jt * Nt + t];
            sv = fmaf(qv.x, iv.x, sv);
            sv = fmaf(-qv.y, iv.y, sv);
          }
          const long long oofs = (b * Cs + c) * chan + pofs;
          if (MODE == EPI_SPECTRAL) {
            a.out[oofs] = sv;
          } else {
            float lin = 0.f;
#pragma unroll
            for (int i = 0; i < CLM; ++i)
              if (i < Cl) lin = fmaf(sW[i * Cs + c], L[i], lin);
            if (MODE == EPI_FWD) {
              a.out[oofs] = gelu_f(sv + lin + sB[c]);
            } else if (MODE == EPI_DA) {
              const float da = a.dz[oofs] * gelu_grad_f(sv + lin + sB[c]);
              a.out[oofs] = da;
              sD[c * PP + pt] = da;
            } else {
              a.out[oofs] = sv + lin;
            }
          }
        }
        if (MODE == EPI_DA) {
#pragma unroll
          for (int i = 0; i < CLM; ++i)
            if (i < Cl) sX[i * PP + pt] = L[i];
        }
      }
      __syncthreads();
      if (MODE == EPI_DA) {
        const int np = zn * Nt;
        for (int e = tid; e < npair; e += nthr) {
          float acc = 0.f;
          if (e < Cl * Cs) {
            const int i = e / Cs, c = e - i * Cs;
            const float* xr = sX + i * PP;
            const float* dr = sD + c * PP;
            for (int p = 0; p < np; ++p) acc = fmaf(xr[p], dr[p], acc);
          } else {
            const float* dr = sD + (e - Cl * Cs) * PP;
            for (int p = 0; p < np; ++p) acc += dr[p];
          }
          // Kahan-compensated running sum over chunks
          float y = acc - sAcc[npair + e];
          float t = sAcc[e] + y;
          sAcc[npair + e] = (t - sAcc[e]) - y;
          sAcc[e] = t;
        }
        __syncthreads();
      }
    }
  }
  if (MODE == EPI_DA) {
    __syncthreads();
    for (int e = tid; e < npair; e += nthr)
      a.part[(long long)blockIdx.x * npair + e] = sAcc[e] - sAcc[npair + e];
  }
}

template <int MODE, int CLM>
static cudaError_t launch_epi_t(const Dims& d, const EpiArgs& a, int* grid_used, cudaStream_t s) {
  EpiK k;
  k.a = a;
  k.B = d.B;
  k.Nx = d.Nx;
  k.Ny = d.Ny;
  k.Nz = (int)d.Nz;
  k.Nt = (int)d.Nt;
  k.Jz = (int)d.Jz;
  k.Jt = (int)d.Jt;
  k.zc = epi_zc(d);
  size_t smem = epilogue_smem_bytes(d, MODE, a.Cs, a.Cl);
  const void* kern = (const void*)k_epi_f32<MODE, CLM>;
  cudaError_t e = allow_smem(kern, smem);
  if (e != cudaSuccess) return e;
  int64_t ncol = d.B * d.Nx * d.Ny;
  int grid = persistent_grid(kern, 256, smem, ncol);
  if (grid > epilogue_max_grid()) grid = epilogue_max_grid();
  if (grid_used) *grid_used = grid;
  static const char* names[4] = {"fno_epi_spectral_f32", "fno_epi_fwd_f32", "fno_epi_da_f32",
                                 "fno_epi_dx_f32"};
  FNO_LAUNCH(names[MODE], (k_epi_f32<MODE, CLM>), grid, 256, smem, s, k);
  return cudaSuccess;
}

template <int MODE>
static cudaError_t launch_epi_m(const Dims& d, const EpiArgs& a, int* g, cudaStream_t s) {
  if (MODE == EPI_SPECTRAL) return launch_epi_t<MODE, 1>(d, a, g, s);
  if (a.Cl <= 8) return launch_epi_t<MODE, 8>(d, a, g, s);
  if (a.Cl <= 16) return launch_epi_t<MODE, 16>(d, a, g, s);
  if (a.Cl <= 32) return launch_epi_t<MODE, 32>(d, a, g, s);
  return launch_epi_t<MODE, 64>(d, a, g, s);
}

cudaError_t launch_epilogue_f32(const Dims& d, const EpiArgs& a, int* grid_used, cudaStream_t s) {
  if (d.B <= 0) {
    if (grid_used) *grid_used = 0;
    return cudaSuccess;
  }
  switch (a.mode) {
    case EPI_SPECTRAL: return launch_epi_m<EPI_SPECTRAL>(d, a, grid_used, s);
    case EPI_FWD: return launch_epi_m<EPI_FWD>(d, a, grid_used, s);
    case EPI_DA: return launch_epi_m<EPI_DA>(d, a, grid_used, s);
    default: return launch_epi_m<EPI_DX>(d, a, grid_used, s);
  }
}

// ---------------------------------------------------------------------------
// Final reduction of the per-CTA partial sums (Kahan-compensated, fixed order)
// and a zero fill.
// ---------------------------------------------------------------------------
__global__ void k_reduce_parts(const float* __restrict__ part, int rows, int npair, int CiCo,
                               float* __restrict__ dwl, float* __restrict__ db) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npair) return;
  float sum = 0.f, comp = 0.f;
  for (int r = 0; r < rows; ++r) {
    float y = part[(long long)r * npair + e] - comp;
    float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
  }
  if (e < CiCo)
    dwl[e] = sum;
  else
    db[e - CiCo] = sum;
}

cudaError_t launch_reduce_partials(const float* part, int rows, int Ci, int Co, float* dwl,
                                   float* db, cudaStream_t s) {
  const int npair = Ci * Co + Co;
  FNO_LAUNCH("fno_reduce_partials", k_reduce_parts, (npair + 127) / 128, 128, 0, s, part, rows,
             npair, Ci * Co, dwl, db);
  return cudaSuccess;
}

__global__ void k_fill_zero(float* __restrict__ p, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = 0.f;
}

cudaError_t launch_fill_zero(float* p, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  FNO_LAUNCH("fno_fill_zero", k_fill_zero, blocks, 256, 0, s, p, (long long)n);
  return cudaSuccess;
}

}  // namespace fno
