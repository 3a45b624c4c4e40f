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
// Spectral convolution and its adjoint (FP32 complex multiply-adds).
//   forward  yh[b][o][j]  = sum_i xh[b][i][j] w[i][o][j]
//   adjoint  gxh[b][i][j] = sum_o conj(w[i][o][j]) g[b][o][j]
//            dw[i][o][j]  = sum_b conj(xh[b][i][j]) g[b][o][j]
// A CTA owns a tile of kMixJ consecutive modes.  It stages the tile's spectra
// for a chunk of BC batch entries in shared memory (rows of kMixJ complex
// values: 128-byte coalesced loads), then each thread keeps one mode j of the
// tile (lane % kMixJ) and walks the output channels of its group (tid / kMixJ,
// stride kMixG), reading the weights straight from HBM in coalesced 128-byte
// rows.  W, dW and the outputs cross HBM once per batch chunk (once when
// B <= BC), and every sum runs in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kMixJ = 16;                   // modes per tile
constexpr int kMixThreads = 256;
constexpr int kMixG = kMixThreads / kMixJ;  // channel groups per tile

__device__ __forceinline__ void cmac(float2& acc, const float2 a, const float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) b
__device__ __forceinline__ void cmac_conj(float2& acc, const float2 a, const float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}

// stage src[b0 + q][c][j0 .. j0 + kMixJ) for q < nb, c < C into dst[q][c][kMixJ]
__device__ __forceinline__ void mix_stage(float2* dst, const float2* __restrict__ src, int b0,
                                          int nb, int BC, int C, long long Mk, long long j0) {
  for (int e = threadIdx.x; e < BC * C * kMixJ; e += kMixThreads) {
    const int jl = e % kMixJ, c = (e / kMixJ) % C, q = e / (kMixJ * C);
    const long long j = j0 + jl;
    dst[e] = (q < nb && j < Mk) ? src[((long long)(b0 + q) * C + c) * Mk + j]
                                : make_float2(0.f, 0.f);
  }
}

template <int BC>
__global__ void __launch_bounds__(kMixThreads)
    k_mix_f32(const float2* __restrict__ xh, const float2* __restrict__ w, float2* __restrict__ yh,
              int B, int Ci, int Co, long long Mk) {
  extern __shared__ float2 mix_sm[];
  float2* xs = mix_sm;  // [BC][Ci][kMixJ]
  const int jl = threadIdx.x % kMixJ, grp = threadIdx.x / kMixJ;
  const long long j0 = (long long)blockIdx.x * kMixJ, j = j0 + jl;
  const bool inj = j < Mk;
  for (int b0 = 0; b0 < B; b0 += BC) {
    const int nb = min(BC, B - b0);
    __syncthreads();
    mix_stage(xs, xh, b0, nb, BC, Ci, Mk, j0);
    __syncthreads();
    if (!inj) continue;
    for (int o = grp; o < Co; o += kMixG) {
      float2 acc[BC];
#pragma unroll
      for (int q = 0; q < BC; ++q) acc[q] = make_float2(0.f, 0.f);
      const float2* wp = w + (long long)o * Mk + j;
#pragma unroll 4
      for (int i = 0; i < Ci; ++i) {
        const float2 wv = __ldg(wp + (long long)i * Co * Mk);
#pragma unroll
        for (int q = 0; q < BC; ++q) cmac(acc[q], xs[(q * Ci + i) * kMixJ + jl], wv);
      }
#pragma unroll
      for (int q = 0; q < BC; ++q)
        if (q < nb) yh[((long long)(b0 + q) * Co + o) * Mk + j] = acc[q];
    }
  }
}

template <int BC>
__global__ void __launch_bounds__(kMixThreads)
    k_mix_adj_f32(const float2* __restrict__ xh, const float2* __restrict__ w,
                  const float2* __restrict__ g, float2* __restrict__ dw, float2* __restrict__ gxh,
                  int B, int Ci, int Co, long long Mk) {
  extern __shared__ float2 mix_sm[];
  float2* xs = mix_sm;                   // [BC][Ci][kMixJ]
  float2* gs = mix_sm + BC * Ci * kMixJ; // [BC][Co][kMixJ]
  const int jl = threadIdx.x % kMixJ, grp = threadIdx.x / kMixJ;
  const long long j0 = (long long)blockIdx.x * kMixJ, j = j0 + jl;
  const bool inj = j < Mk;
  for (int b0 = 0; b0 < B; b0 += BC) {
    const int nb = min(BC, B - b0);
    __syncthreads();
    if (dw) mix_stage(xs, xh, b0, nb, BC, Ci, Mk, j0);
    mix_stage(gs, g, b0, nb, BC, Co, Mk, j0);
    __syncthreads();
    if (!inj) continue;
    if (gxh) {
      for (int i = grp; i < Ci; i += kMixG) {
        float2 ga[BC];
#pragma unroll
        for (int q = 0; q < BC; ++q) ga[q] = make_float2(0.f, 0.f);
        const float2* wp = w + (long long)i * Co * Mk + j;
#pragma unroll 8
        for (int o = 0; o < Co; ++o) {
          const float2 wv = __ldg(wp + (long long)o * Mk);
#pragma unroll
          for (int q = 0; q < BC; ++q) cmac_conj(ga[q], wv, gs[(q * Co + o) * kMixJ + jl]);
        }
#pragma unroll
        for (int q = 0; q < BC; ++q)
          if (q < nb) gxh[((long long)(b0 + q) * Ci + i) * Mk + j] = ga[q];
      }
    }
    if (dw) {
      for (int i = 0; i < Ci; ++i) {
        float2 xv[BC];
#pragma unroll
        for (int q = 0; q < BC; ++q) xv[q] = xs[(q * Ci + i) * kMixJ + jl];
        for (int o = grp; o < Co; o += kMixG) {
          float2 da = make_float2(0.f, 0.f);
#pragma unroll
          for (int q = 0; q < BC; ++q) cmac_conj(da, xv[q], gs[(q * Co + o) * kMixJ + jl]);
          float2* dp = dw + ((long long)i * Co + o) * Mk + j;
          if (b0 == 0) {
            *dp = da;
          } else {
            const float2 p = *dp;
            *dp = make_float2(p.x + da.x, p.y + da.y);
          }
        }
      }
    }
  }
}

static int mix_bc(int64_t B) { return B <= 1 ? 1 : B <= 2 ? 2 : B <= 4 ? 4 : 8; }

template <int BC>
static cudaError_t launch_mix_bc(const Dims& d, const float2* xh, const float2* w, float2* yh,
                                 cudaStream_t s) {
  const size_t smem = sizeof(float2) * (size_t)BC * (size_t)d.Ci * kMixJ;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_mix_f32<BC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const unsigned grid = (unsigned)((d.Mk + kMixJ - 1) / kMixJ);
  FNO_LAUNCH("fno_mix_f32", k_mix_f32<BC>, grid, kMixThreads, smem, s, xh, w, yh, (int)d.B,
             (int)d.Ci, (int)d.Co, (long long)d.Mk);
  return cudaSuccess;
}

template <int BC>
static cudaError_t launch_mix_adj_bc(const Dims& d, const float2* xh, const float2* w,
                                     const float2* g, float2* dw, float2* gxh, cudaStream_t s) {
  const size_t smem = sizeof(float2) * (size_t)BC * (size_t)(d.Ci + d.Co) * kMixJ;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_mix_adj_f32<BC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const unsigned grid = (unsigned)((d.Mk + kMixJ - 1) / kMixJ);
  FNO_LAUNCH("fno_mix_adjoint_f32", k_mix_adj_f32<BC>, grid, kMixThreads, smem, s, xh, w, g, dw,
             gxh, (int)d.B, (int)d.Ci, (int)d.Co, (long long)d.Mk);
  return cudaSuccess;
}

cudaError_t launch_mix_f32(const Dims& d, const float2* xh, const float2* w, float2* yh,
                           cudaStream_t s) {
  if (d.B <= 0) return cudaSuccess;
  switch (mix_bc(d.B)) {
    case 1: return launch_mix_bc<1>(d, xh, w, yh, s);
    case 2: return launch_mix_bc<2>(d, xh, w, yh, s);
    case 4: return launch_mix_bc<4>(d, xh, w, yh, s);
    default: return launch_mix_bc<8>(d, xh, w, yh, s);
  }
}

cudaError_t launch_mix_adjoint_f32(const Dims& d, const float2* xh, const float2* w,
                                   const float2* g, float2* dw, float2* gxh, cudaStream_t s) {
  if (d.B <= 0) return cudaSuccess;
  switch (mix_bc(d.B)) {
    case 1: return launch_mix_adj_bc<1>(d, xh, w, g, dw, gxh, s);
    case 2: return launch_mix_adj_bc<2>(d, xh, w, g, dw, gxh, s);
    case 4: return launch_mix_adj_bc<4>(d, xh, w, g, dw, gxh, s);
    default: return launch_mix_adj_bc<8>(d, xh, w, g, dw, gxh, s);
  }
}

// ---------------------------------------------------------------------------
// Inverse z, t stages fused with the pointwise epilogue (FP32 CUDA cores).
// A 128-thread CTA walks a contiguous range of tiles; a tile is P = 128
// consecutive points (z, t) of one (b, x, y) column (fewer at the column's
// end) and all its channels, one thread per point.  When Nt divides 128 a
// tile is 128 / Nt whole z-planes; otherwise it starts and ends inside planes
// and touches at most ZM = 1 + ceil(127 / Nt) of them.
//   Q[zz][jt][o] = inverse z stage of the column spectrum, with +-k pairing:
//       Q(z) = sum_{k=0..mz} E_k cos(k th) + i sum_{k=1..mz} O_k sin(k th)
//       E_0 = U_0, E_k = U_k + U_-k, O_k = U_k - U_-k, E_mz = U_-mz, O_mz = -U_-mz
//   per point and 4 outputs at a time (shared-memory vector broadcasts):
//       A_o = bias_o + sum_jt (Qr[jt][o] c_jt(t) - Qi[jt][o] s_jt(t)) + sum_i W(i, o) L_i
//   SPECTRAL: out = A (no bias, no linear term)   FWD: out = GELU(A)
//   DA: out = dA = dz GELU'(A), and dW_lin / db partial sums   DX: out = A
// ---------------------------------------------------------------------------
struct EpiK {
  EpiArgs a;
  long long NxNy, ntiles;
  long long nzc;        // tiles per column: ceil(Nz * Nt / 128)
  int Nz, Nt, Jz, Jt, mz;
  int ZM;               // z-planes a tile touches at most
  int P;                // points per tile, min(128, Nz * Nt)
  int CS4;
  int IB, OB, KG;       // EPI_DA: 4x4 (i, o) blocks of dW_lin, point groups
  int CLW;              // weight rows held in shared memory (the template's channel bound)
  uint32_t off[8];      // shared-memory region offsets (16-byte aligned)
};

constexpr int kEpiP = 128;  // points per tile (one per thread)

// points per tile and the most z-planes a tile touches
static int epi_points(const Dims& d) { return (int)std::min<int64_t>(kEpiP, d.Nz * d.Nt); }
static int epi_planes(const Dims& d) {
  int64_t zm = (kEpiP % d.Nt == 0) ? kEpiP / d.Nt : 1 + (kEpiP - 1 + d.Nt - 1) / d.Nt;
  return (int)std::min<int64_t>(zm, d.Nz);
}

// channel bound of the lin-input register array (template CLM) for Cl channels
static int epi_clm(int Cl) {
  if (Cl <= 0) return 0;
  static const int b[] = {4, 8, 12, 16, 20, 24, 32, 48, 64};
  for (int v : b)
    if (Cl <= v) return v;
  return 64;
}

static void epi_layout(const Dims& d, int mode, int Cs, int Cl, size_t off[8], size_t& total) {
  const int ZM = epi_planes(d);
  const int P = epi_points(d);
  const int CS4 = (Cs + 3) / 4 * 4;
  auto al = [](size_t x) { return (x + 15) / 16 * 16; };
  size_t o = 0;
  off[0] = o;  // eo: [Cs][Jt][mz+1] float4
  o = al(o + sizeof(float4) * (size_t)(Cs * d.Jt * (d.mz + 1)));
  off[1] = o;  // cs: [Nz][mz+1] float2
  o = al(o + sizeof(float2) * (size_t)(d.Nz * (d.mz + 1)));
  off[2] = o;  // qs: [ZM][Jt][2][CS4] float
  o = al(o + sizeof(float) * (size_t)(ZM * d.Jt * 2 * CS4));
  off[3] = o;  // w: [CLW][CS4], CLW = Cl rounded up to the kernel's channel bound
  o = al(o + sizeof(float) * (size_t)(epi_clm(Cl) * CS4));
  off[4] = o;  // bias: [CS4]
  o = al(o + sizeof(float) * (size_t)CS4);
  off[5] = o;  // DA: x tile [Cl][P+1]
  if (mode == EPI_DA) o = al(o + sizeof(float) * (size_t)(Cl * (P + 1)));
  off[6] = o;  // DA: dA tile [CS4][P+1]
  if (mode == EPI_DA) o = al(o + sizeof(float) * (size_t)(CS4 * (P + 1)));
  // DA: Kahan (sum, compensation) pairs [IB*OB - 128][2][16] of the 4x4 (i, o)
  // blocks beyond the first 128 (each thread keeps its first block in
  // registers).  Placed past the first 8 KB, which the final reduction reuses
  // for the register-held sums.
  if (mode == EPI_DA) o = std::max(o, (size_t)(128 * 16 * sizeof(float)));
  off[7] = o;
  if (mode == EPI_DA) {
    const int nblk = ((Cl + 1 + 3) / 4) * (CS4 / 4);
    if (nblk > 128) o = al(o + sizeof(float) * 32 * (size_t)(nblk - 128));
  }
  total = o;
}

size_t epilogue_smem_bytes(const Dims& d, int mode, int Cs, int Cl) {
  size_t off[8], total;
  epi_layout(d, mode, Cs, Cl, off, total);
  // in DA mode the final reduction reuses the first 8 KB (128 items x 16
  // sums), which epi_layout already keeps below the spill region
  return total;
}

int epilogue_max_grid() { return 1024; }

template <int MODE, int CLM, int JTM>
__global__ void __launch_bounds__(128, 4) k_epi_f32(const EpiK k) {
  extern __shared__ float4 smem4[];
  const EpiArgs& a = k.a;
  const int Cs = a.Cs, Cl = (MODE == EPI_SPECTRAL) ? 0 : a.Cl;
  const int Jz = k.Jz, Jt = k.Jt, Nz = k.Nz, Nt = k.Nt, mz = k.mz, P = k.P, CS4 = k.CS4;
  const int PP = P + 1;
  unsigned char* base = reinterpret_cast<unsigned char*>(smem4);
  float4* eo = reinterpret_cast<float4*>(base + k.off[0]);
  float2* cs = reinterpret_cast<float2*>(base + k.off[1]);
  float* qs = reinterpret_cast<float*>(base + k.off[2]);
  float* sw = reinterpret_cast<float*>(base + k.off[3]);
  float* sbias = reinterpret_cast<float*>(base + k.off[4]);
  float* sx = reinterpret_cast<float*>(base + k.off[5]);
  float* sda = reinterpret_cast<float*>(base + k.off[6]);
  const int tid = threadIdx.x;

  for (int e = tid; e < Nz * (mz + 1); e += 128) {
    const int z = e / (mz + 1), kk = e - z * (mz + 1);
    const float2 f = a.Iz[z * Jz + kk];  // jz = kk: kz = kk (kk < mz), kz = -mz (kk = mz)
    cs[e] = (kk < mz) ? f : make_float2(f.x, -f.y);
  }
  if (MODE != EPI_SPECTRAL) {
    for (int e = tid; e < k.CLW * CS4; e += 128) {
      const int i = e / CS4, c = e - i * CS4;
      sw[e] = (c < Cs && i < Cl) ? a.wlin[(long long)i * a.w_si + (long long)c * a.w_sc] : 0.f;
    }
  }
  for (int c = tid; c < CS4; c += 128)
    sbias[c] = ((MODE == EPI_FWD || MODE == EPI_DA) && c < Cs) ? a.bias[c] : 0.f;

  // this thread's point is p of each tile; its t (and so the inverse-t
  // factors) changes between tiles only when Nt does not divide 128
  const int p = tid;
  int cur_t = -1;
  float itr[JTM], iti[JTM];

  // EPI_DA: work items are (4x4 block of (i, o), point group) pairs, item
  // it = g * nblk + block.  KG point groups split the points when there are
  // fewer than 128 blocks; with more (KG = 1), a thread owns blocks tid,
  // tid + 128, ...  Its first item's Kahan running sums live in registers, the
  // others' in shared memory (racc).
  const int nblk = k.IB * k.OB;
  const int nitem = nblk * k.KG;
  const bool wthread = (MODE == EPI_DA) && tid < nitem;
  float* racc = reinterpret_cast<float*>(base + k.off[7]);
  if (MODE == EPI_DA)
    for (int e = tid; e < (nitem - 128) * 32; e += 128) racc[e] = 0.f;
  float wsum[16], wcmp[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    wsum[q] = 0.f;
    wcmp[q] = 0.f;
  }

  const long long plane = (long long)Nz * Nt;
  const long long chan = k.NxNy * plane;
  const long long t_begin = k.ntiles * blockIdx.x / gridDim.x;
  const long long t_end = k.ntiles * (blockIdx.x + 1) / gridDim.x;
  long long cur_col = -1;
  for (long long tau = t_begin; tau < t_end; ++tau) {
    const long long col = tau / k.nzc;
    const long long s0 = (tau - col * k.nzc) * kEpiP;  // first point of the tile in the column
    const int valid = (int)min((long long)kEpiP, plane - s0);
    const int z0 = (int)(s0 / Nt);                      // first plane the tile touches
    const int tf = (int)(s0 - (long long)z0 * Nt);      // its first point's t
    const int zn = (tf + valid - 1) / Nt + 1;           // planes touched, <= ZM
    const long long b = col / k.NxNy, xy = col - b * k.NxNy;
    const int zz_p = (tf + p) / Nt, t = (tf + p) - zz_p * Nt;
    if (t != cur_t) {
#pragma unroll
      for (int jt = 0; jt < JTM; ++jt) {
        if (jt < Jt) {
          const float2 f = __ldg(a.It + jt * Nt + t);
          itr[jt] = f.x;
          iti[jt] = -f.y;
        } else {
          itr[jt] = 0.f;
          iti[jt] = 0.f;
        }
      }
      cur_t = t;
    }
    __syncthreads();  // previous tile's shared-memory reads are done
    if (col != cur_col) {
      const int JZT = Jz * Jt;
      const int neo = Cs * Jt * (mz + 1);
      for (int e0 = tid; e0 < neo; e0 += 4 * 128) {
        float2 av[4], mv[4];
#pragma unroll
        for (int u4 = 0; u4 < 4; ++u4) {
          const int e = e0 + u4 * 128;
          av[u4] = make_float2(0.f, 0.f);
          mv[u4] = make_float2(0.f, 0.f);
          if (e < neo) {
            const int kk = e % (mz + 1), jt = (e / (mz + 1)) % Jt, c = e / ((mz + 1) * Jt);
            const float2* u = a.U + ((b * Cs + c) * k.NxNy + xy) * JZT + jt;
            if (kk < mz) av[u4] = __ldg(u + kk * Jt);
            if (kk > 0) mv[u4] = __ldg(u + (2 * mz - kk) * Jt);
          }
        }
#pragma unroll
        for (int u4 = 0; u4 < 4; ++u4) {
          const int e = e0 + u4 * 128;
          if (e < neo) {
            const float2 av_ = av[u4], mv_ = mv[u4];
            eo[e] = make_float4(av_.x + mv_.x, av_.y + mv_.y, av_.x - mv_.x, av_.y - mv_.y);
          }
        }
      }
      cur_col = col;
      __syncthreads();
    }
    // lin inputs of this point (issued early; consumed after Q is ready)
    float x[CLM > 0 ? CLM : 1];
    const long long pofs = xy * plane + s0 + p;
    const bool pv = p < valid;
    if (MODE != EPI_SPECTRAL) {
      const float* xp = a.lin_in + (b * Cl) * chan + pofs;
#pragma unroll
      for (int i = 0; i < CLM; ++i) x[i] = (i < Cl && pv) ? __ldg(xp + (long long)i * chan) : 0.f;
    }
    // Q of this tile's planes: one (o, jt, zz) unit per step
    {
      const int units = Cs * Jt * zn;
      for (int e = tid; e < units; e += 128) {
        const int zz = e % zn, cj = e / zn;
        const int jt = cj % Jt, c = cj / Jt;
        const float4* src = eo + (size_t)(c * Jt + jt) * (mz + 1);
        const float2* cz = cs + (size_t)(z0 + zz) * (mz + 1);
        float qr = 0.f, qi = 0.f, qr2 = 0.f, qi2 = 0.f;
        int kk = 0;
        for (; kk + 1 <= mz; kk += 2) {
          const float4 r0 = src[kk], r1 = src[kk + 1];
          const float2 t0 = cz[kk], t1 = cz[kk + 1];
          qr = fmaf(r0.x, t0.x, qr);
          qr = fmaf(-r0.w, t0.y, qr);
          qi = fmaf(r0.y, t0.x, qi);
          qi = fmaf(r0.z, t0.y, qi);
          qr2 = fmaf(r1.x, t1.x, qr2);
          qr2 = fmaf(-r1.w, t1.y, qr2);
          qi2 = fmaf(r1.y, t1.x, qi2);
          qi2 = fmaf(r1.z, t1.y, qi2);
        }
        if (kk <= mz) {
          const float4 r0 = src[kk];
          const float2 t0 = cz[kk];
          qr = fmaf(r0.x, t0.x, qr);
          qr = fmaf(-r0.w, t0.y, qr);
          qi = fmaf(r0.y, t0.x, qi);
          qi = fmaf(r0.z, t0.y, qi);
        }
        float* qd = qs + ((size_t)(zz * Jt + jt) * 2) * CS4 + c;
        qd[0] = qr + qr2;
        qd[CS4] = qi + qi2;
      }
      // zero the padded output columns once per tile (read by the vector loads)
      for (int e = tid; e < zn * Jt * 2 * (CS4 - Cs); e += 128) {
        const int c = Cs + e % (CS4 - Cs), r = e / (CS4 - Cs);
        qs[(size_t)r * CS4 + c] = 0.f;
      }
    }
    __syncthreads();
    // per point: 4 outputs at a time (only threads that own a point of this tile)
    if (pv) {
      const float* qp = qs + (size_t)(zz_p * Jt) * 2 * CS4;
      float* optr = a.out + (b * Cs) * chan + pofs;
      const float* dzp = (MODE == EPI_DA) ? a.dz + (b * Cs) * chan + pofs : nullptr;
      for (int c0 = 0; c0 < Cs; c0 += 4) {
        float dzq[4];
        if (MODE == EPI_DA) {
#pragma unroll
          for (int q = 0; q < 4; ++q) dzq[q] = (c0 + q < Cs) ? __ldg(dzp + (long long)(c0 + q) * chan) : 0.f;
        }
        float4 acc = *reinterpret_cast<const float4*>(sbias + c0);
#pragma unroll
        for (int jt = 0; jt < JTM; ++jt) {
          if (jt < Jt) {
            const float4 qr = *reinterpret_cast<const float4*>(qp + (size_t)(jt * 2) * CS4 + c0);
            const float4 qi = *reinterpret_cast<const float4*>(qp + (size_t)(jt * 2 + 1) * CS4 + c0);
            acc.x = fmaf(qr.x, itr[jt], fmaf(qi.x, iti[jt], acc.x));
            acc.y = fmaf(qr.y, itr[jt], fmaf(qi.y, iti[jt], acc.y));
            acc.z = fmaf(qr.z, itr[jt], fmaf(qi.z, iti[jt], acc.z));
            acc.w = fmaf(qr.w, itr[jt], fmaf(qi.w, iti[jt], acc.w));
          }
        }
        if (MODE != EPI_SPECTRAL) {
          const float* wp = sw + c0;
#pragma unroll
          for (int i = 0; i < CLM; ++i) {
            const float4 w4 = *reinterpret_cast<const float4*>(wp + (size_t)i * CS4);
            acc.x = fmaf(w4.x, x[i], acc.x);
            acc.y = fmaf(w4.y, x[i], acc.y);
            acc.z = fmaf(w4.z, x[i], acc.z);
            acc.w = fmaf(w4.w, x[i], acc.w);
          }
        }
        const float av[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = c0 + q;
          if (c < Cs) {
            float* o = optr + (long long)c * chan;
            if (MODE == EPI_FWD) {
              *o = gelu_f(av[q]);
              if (a.gp) a.gp[o - a.out] = gelu_grad_f(av[q]);  // training forward
            } else if (MODE == EPI_DA) {
              const float da = dzq[q] * gelu_grad_f(av[q]);
              *o = da;
              sda[c * PP + p] = da;
            } else {
              *o = av[q];
            }
          } else if (MODE == EPI_DA && c < CS4) {
            sda[c * PP + p] = 0.f;
          }
        }
      }
    }
    if (MODE == EPI_DA) {
      if (p < P) {
        if (!pv)
          for (int c = 0; c < CS4; ++c) sda[c * PP + p] = 0.f;
#pragma unroll
        for (int i = 0; i < CLM; ++i)
          if (i < Cl) sx[i * PP + p] = x[i];
      }
      __syncthreads();
      if (wthread) {
        for (int it = tid; it < nitem; it += 128) {
          const int bl = it % nblk, kg = it / nblk;
          const int i0 = (bl / k.OB) * 4, o0w = (bl % k.OB) * 4;
          const int pa = kg * P / k.KG, pb = min((kg + 1) * P / k.KG, valid);
          float part[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) part[q] = 0.f;
          for (int pt = pa; pt < pb; ++pt) {
            float xv[4], dv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int i = i0 + u;
              xv[u] = i < Cl ? sx[i * PP + pt] : (i == Cl ? 1.f : 0.f);
              dv[u] = sda[(o0w + u) * PP + pt];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) part[u * 4 + v] = fmaf(xv[u], dv[v], part[u * 4 + v]);
          }
          if (it < 128) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const float y = part[q] - wcmp[q];
              const float s = wsum[q] + y;
              wcmp[q] = (s - wsum[q]) - y;
              wsum[q] = s;
            }
          } else {
            float* r = racc + (it - 128) * 32;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const float y = part[q] - r[16 + q];
              const float s = r[q] + y;
              r[16 + q] = (s - r[q]) - y;
              r[q] = s;
            }
          }
        }
      }
    }
  }
  if (MODE == EPI_DA) {
    __syncthreads();
    float* red = reinterpret_cast<float*>(base);
    if (wthread) {
#pragma unroll
      for (int q = 0; q < 16; ++q) red[tid * 16 + q] = wsum[q] - wcmp[q];
    }
    __syncthreads();
    const int npair = Cl * Cs + Cs;
    for (int e = tid; e < nblk * 16; e += 128) {
      const int bl = e / 16, q = e % 16;
      const int i = (bl / k.OB) * 4 + q / 4, c = (bl % k.OB) * 4 + q % 4;
      float s = 0.f, comp = 0.f;
      for (int g = 0; g < k.KG; ++g) {
        const int it = g * nblk + bl;
        const float v = it < 128 ? red[it * 16 + q]
                                 : racc[(it - 128) * 32 + q] - racc[(it - 128) * 32 + 16 + q];
        const float y = v - comp;
        const float tt = s + y;
        comp = (tt - s) - y;
        s = tt;
      }
      if (c < Cs && i <= Cl) {
        const int idx = (i < Cl) ? i * Cs + c : Cl * Cs + c;
        a.part[(long long)blockIdx.x * npair + idx] = s;
      }
    }
  }
}

template <int MODE, int CLM, int JTM>
static cudaError_t launch_epi_t(const Dims& d, const EpiArgs& a, int* grid_used, cudaStream_t s) {
  EpiK k{};
  k.a = a;
  k.NxNy = d.Nx * d.Ny;
  k.Nz = (int)d.Nz;
  k.Nt = (int)d.Nt;
  k.Jz = (int)d.Jz;
  k.Jt = (int)d.Jt;
  k.mz = (int)d.mz;
  k.ZM = epi_planes(d);
  k.P = epi_points(d);
  k.nzc = (d.Nz * d.Nt + kEpiP - 1) / kEpiP;
  k.CS4 = (a.Cs + 3) / 4 * 4;
  const int Cl = MODE == EPI_SPECTRAL ? 0 : a.Cl;
  k.IB = (Cl + 1 + 3) / 4;
  k.OB = k.CS4 / 4;
  k.KG = std::max(1, 128 / (k.IB * k.OB));
  k.CLW = epi_clm(Cl);
  k.ntiles = d.B * d.Nx * d.Ny * (long long)k.nzc;
  {
    size_t off[8], total;
    epi_layout(d, MODE, a.Cs, Cl, off, total);
    for (int q = 0; q < 8; ++q) k.off[q] = (uint32_t)off[q];
  }
  const size_t smem = epilogue_smem_bytes(d, MODE, a.Cs, Cl);
  const void* kern = (const void*)k_epi_f32<MODE, CLM, JTM>;
  cudaError_t e = allow_smem(kern, smem);
  if (e != cudaSuccess) return e;
  int grid = persistent_grid(kern, 128, smem, k.ntiles);
  if (grid > epilogue_max_grid()) grid = epilogue_max_grid();
  if (grid_used) *grid_used = grid;
  static const char* names[4] = {"fno_epi_spectral_f32", "fno_epi_fwd_f32", "fno_epi_da_f32",
                                 "fno_epi_dx_f32"};
  // the forward of a training step also stores GELU'(A)
  const char* name = (MODE == EPI_FWD && a.gp) ? "fno_epi_fwd_train_f32" : names[MODE];
  FNO_LAUNCH(name, (k_epi_f32<MODE, CLM, JTM>), grid, 128, smem, s, k);
  return cudaSuccess;
}

template <int MODE, int JTM>
static cudaError_t launch_epi_j(const Dims& d, const EpiArgs& a, int* g, cudaStream_t s) {
  if constexpr (MODE == EPI_SPECTRAL) {
    return launch_epi_t<MODE, 0, JTM>(d, a, g, s);
  } else {
  switch (epi_clm(a.Cl)) {
    case 4: return launch_epi_t<MODE, 4, JTM>(d, a, g, s);
    case 8: return launch_epi_t<MODE, 8, JTM>(d, a, g, s);
    case 12: return launch_epi_t<MODE, 12, JTM>(d, a, g, s);
    case 16: return launch_epi_t<MODE, 16, JTM>(d, a, g, s);
    case 20: return launch_epi_t<MODE, 20, JTM>(d, a, g, s);
    case 24: return launch_epi_t<MODE, 24, JTM>(d, a, g, s);
    case 32: return launch_epi_t<MODE, 32, JTM>(d, a, g, s);
    case 48: return launch_epi_t<MODE, 48, JTM>(d, a, g, s);
    default: return launch_epi_t<MODE, 64, JTM>(d, a, g, s);
  }
  }
}

template <int MODE>
static cudaError_t launch_epi_m(const Dims& d, const EpiArgs& a, int* g, cudaStream_t s) {
  if (d.Jt <= 8) return launch_epi_j<MODE, 8>(d, a, g, s);
  return launch_epi_j<MODE, 16>(d, a, g, s);
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
