// fno_tc.cu -- tensor-core (tcgen05 / TMEM) kernels of the two stages that
// carry the block's full-size traffic:
//
//   k_fwd_tz_tc  the pruned forward DFT over t then z of every (b, c, x, y)
//                column (the first half of F_yzt, S_yzt in Alg. 2), as two
//                chained GEMMs per group of columns:
//                  t stage  D1[(col,z)][(jt,ri)]  = X[(col,z)][t]  . Ft[(jt,ri)][t]
//                  z stage  D2[(col,jt)][(jz,ri)] = P[(col,jt)][(ri',z)] . Fz'[(jz,ri)][(ri',z)]
//                X tiles arrive by bulk copy (TMA engine) into a ring, are split to
//                BF16 hi/lo in shared memory, and D1 is moved TMEM -> registers ->
//                shared memory (transposed) to become the z-stage operand.
//
//   k_epi_tc     the inverse z, t stages fused with the pointwise 1x1 linear, bias
//                and GELU (or their gradients).  For a tile of 128 grid points of
//                one (b, x, y) column the pre-activation is one GEMM
//                  D[p][o] = sum_i X[p][i] Wl[i][o]
//                          + sum_zz sum_(jt,ri) It'[t(p)][(jt,ri)] [z(p) = zz] Q[zz][(jt,ri)][o]
//                where Q = inverse z stage of the column's spectrum (CUDA cores) and
//                It' the inverse t basis.  The zz-banded t basis is read through
//                shifted descriptor windows of one zero-padded buffer.
//
// Precision: BF16 operands (one product) or split BF16 (x = hi + lo, products
// hi.hi + hi.lo + lo.hi), FP32 accumulation in TMEM.  Every wait is bounded; on
// timeout the kernel raises *err, drains what it started and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>

#include "fno_internal.h"
#include "umma.h"

namespace fno {

using namespace umma;

#define FNO_LAUNCH_TC(name, kern, grid, block, smem, stream, ...) \
  do {                                                            \
    prof_before(name, stream);                                    \
    kern<<<grid, block, smem, stream>>>(__VA_ARGS__);             \
    cudaError_t e_ = cudaGetLastError();                          \
    prof_after(stream);                                           \
    if (e_ != cudaSuccess) return e_;                             \
  } while (0)

// ---- small helpers ------------------------------------------------------------
__device__ __forceinline__ uint32_t bf2(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  float2 hf = __bfloat1622float2(h);
  __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<uint32_t*>(&h);
  lo = *reinterpret_cast<uint32_t*>(&l);
}
__device__ __forceinline__ void split1(float a, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(a);
  lo = __float2bfloat16_rn(a - __bfloat162float(hi));
}
// byte offset of element (r, k) of a 2-byte K-major no-swizzle operand
__device__ __forceinline__ uint32_t koff(uint32_t r, uint32_t k, uint32_t sbo, uint32_t lbo) {
  return (r & 7u) * 16u + (r >> 3) * sbo + (k & 7u) * 2u + (k >> 3) * lbo;
}
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
}

static uint32_t pow2_cols(uint32_t n) {
  uint32_t c = 32;
  while (c < n) c <<= 1;
  return c;
}
static uint32_t up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

static const long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz per wait

// ============================================================================
// Forward t, z stages
// ============================================================================
struct FwdTcK {
  const float* in;
  float2* out;
  const float2* Ft;  // [Jt][Nt]
  const float2* Fz;  // [Jz][Nz]
  int* err;
  long long ncol;     // columns (b, c, x, y)
  long long ngroups;  // groups of G columns
  int Nz, Nt, Jz, Jt;
  int cpt;  // columns per 128-row t tile (128 / Nz)
  int G;    // columns per z-stage group
  int tpg;  // t tiles per group
  int K1, N1, K2, N2, S;
  uint32_t lbo2, sbo2;       // z-stage A operand strides (padded)
  uint32_t o_xf, xf_bytes;   // ring of fp32 tiles
  uint32_t o_a1, a1_bytes;   // t-stage A operand, 2 buffers x (hi, lo)
  uint32_t o_b1, b1_bytes;   // t basis (hi, lo)
  uint32_t o_a2;             // z-stage A operand (one of hi / lo at a time)
  uint32_t o_b2, b2_bytes;   // z basis (hi, lo)
  uint32_t o_bar;
  uint32_t tmem_cols, d2_col;
};

template <bool SPLIT>
__global__ void __launch_bounds__(160, 1) k_fwd_tz_tc(const FwdTcK p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* xf = sm + p.o_xf;
  unsigned char* a1 = sm + p.o_a1;
  unsigned char* b1 = sm + p.o_b1;
  unsigned char* a2 = sm + p.o_a2;
  unsigned char* b2 = sm + p.o_b2;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + p.o_bar);  // [S]
  uint64_t* empty = full + p.S;                                // [S]
  uint64_t* bar_t = empty + p.S;                               // [2]
  uint64_t* bar_z = bar_t + 2;                                 // [1]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar_z + 1);
  int* sflag = reinterpret_cast<int*>(tslot + 1);
  const int S = p.S, Nz = p.Nz, Nt = p.Nt, Jz = p.Jz, Jt = p.Jt;
  const uint32_t sbo1 = (uint32_t)p.K1 * 16u;  // t-stage operands: K1/8 chunks of 128 B
  const uint32_t sbo_b2 = (uint32_t)p.K2 * 16u;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 128);
    }
    mbar_init(&bar_t[0], 1);
    mbar_init(&bar_t[1], 1);
    mbar_init(&bar_z[0], 1);
    *sflag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, p.tmem_cols);
    tmem_relinquish();
  }
  // constant operands: zero the t-stage A buffers (K padding stays zero), build bases
  for (uint32_t e = tid; e < p.a1_bytes * 4u / 16u; e += blockDim.x)
    reinterpret_cast<uint4*>(a1)[e] = make_uint4(0, 0, 0, 0);
  for (int e = tid; e < p.N1 * p.K1; e += blockDim.x) {
    const int n = e / p.K1, k = e - n * p.K1;
    float v = 0.f;
    if (k < Nt && n < 2 * Jt) {
      const float2 f = p.Ft[(n >> 1) * Nt + k];
      v = (n & 1) ? f.y : f.x;
    }
    __nv_bfloat16 h, l;
    split1(v, h, l);
    const uint32_t off = koff(n, k, sbo1, 128);
    *reinterpret_cast<__nv_bfloat16*>(b1 + off) = h;
    *reinterpret_cast<__nv_bfloat16*>(b1 + p.b1_bytes + off) = l;
  }
  for (int e = tid; e < p.N2 * p.K2; e += blockDim.x) {
    const int n = e / p.K2, k = e - n * p.K2;
    float v = 0.f;
    if (n < 2 * Jz) {
      const int jz = n >> 1, ro = n & 1, ri = k / Nz, z = k - ri * Nz;
      const float2 f = p.Fz[jz * Nz + z];
      // re out: Fr * Pr - Fi * Pi ; im out: Fi * Pr + Fr * Pi
      v = (ro == 0) ? (ri == 0 ? f.x : -f.y) : (ri == 0 ? f.y : f.x);
    }
    __nv_bfloat16 h, l;
    split1(v, h, l);
    const uint32_t off = koff(n, k, sbo_b2, 128);
    *reinterpret_cast<__nv_bfloat16*>(b2 + off) = h;
    *reinterpret_cast<__nv_bfloat16*>(b2 + p.b2_bytes + off) = l;
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t idt = idesc(kFmtBF16, 128, p.N1);
  const uint32_t idz = idesc(kFmtBF16, 128, p.N2);

  if (warp == 4) {
    // ---------------- producer: bulk copies of 128-row tiles ----------------
    if (lane == 0) {
      long long it = 0;
      bool ok = true;
      for (long long g = blockIdx.x; g < p.ngroups && ok; g += gridDim.x) {
        for (int j = 0; j < p.tpg; ++j) {
          const long long tile = g * p.tpg + j;
          const long long col0 = tile * p.cpt;
          if (col0 >= p.ncol) break;
          const long long ncols = min((long long)p.cpt, p.ncol - col0);
          const uint32_t bytes = (uint32_t)(ncols * Nz * Nt * 4);
          const int s = (int)(it % S);
          const uint32_t par = (uint32_t)(((it / S) & 1) ^ 1);
          if (!mbar_wait(&empty[s], par, kWaitCycles)) {
            ok = false;
            atomicExch(p.err, 1);
            break;
          }
          mbar_arrive_expect_tx(&full[s], bytes);
          bulk_g2s(xf + (size_t)s * p.xf_bytes, p.in + col0 * Nz * Nt, bytes, &full[s]);
          ++it;
        }
      }
      // drain: every issued copy must have landed before the CTA may exit
      for (long long k = (it > S ? it - S : 0); k < it; ++k)
        mbar_wait(&full[k % S], (uint32_t)((k / S) & 1), kWaitCycles);
    }
  } else {
    // ---------------- math warps 0..3 ----------------
    long long it = 0;
    uint32_t cnt_t[2] = {0, 0}, cnt_z = 0;
    bool ok = true;
    const int r = tid;  // TMEM lane / tile row of this thread
    for (long long g = blockIdx.x; g < p.ngroups && ok; g += gridDim.x) {
      const long long gcol0 = g * p.G;
      const int gcols = (int)min((long long)p.G, p.ncol - gcol0);
      const int ntile = (gcols + p.cpt - 1) / p.cpt;
      // ---- t stage, one 128-row tile at a time ----
      for (int j = 0; j < ntile; ++j) {
        const int s = (int)(it % S);
        const int bb = (int)(it & 1);
        if (!mbar_wait(&full[s], (uint32_t)((it / S) & 1), kWaitCycles)) ok = false;
        if (cnt_t[bb] > 0 && !mbar_wait(&bar_t[bb], (cnt_t[bb] - 1) & 1, kWaitCycles)) ok = false;
        if (!ok) {
          atomicExch(p.err, 1);
          *sflag = 1;
        }
        fence_after_sync();
        const long long col0 = (g * p.tpg + j) * p.cpt;
        const int rows = (int)min((long long)p.cpt, p.ncol - col0) * Nz;
        const float* xs = reinterpret_cast<const float*>(xf + (size_t)s * p.xf_bytes);
        unsigned char* ah = a1 + (size_t)bb * 2 * p.a1_bytes;
        const int nch = Nt / 8;
        for (int e = tid; e < 128 * nch; e += 128) {
          const int row = e / nch, c8 = e - row * nch;
          float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
          if (row < rows) {
            v0 = reinterpret_cast<const float4*>(xs + row * Nt + c8 * 8)[0];
            v1 = reinterpret_cast<const float4*>(xs + row * Nt + c8 * 8)[1];
          }
          uint4 h, l;
          if (SPLIT) {
            split2(v0.x, v0.y, h.x, l.x);
            split2(v0.z, v0.w, h.y, l.y);
            split2(v1.x, v1.y, h.z, l.z);
            split2(v1.z, v1.w, h.w, l.w);
          } else {
            h = make_uint4(bf2(v0.x, v0.y), bf2(v0.z, v0.w), bf2(v1.x, v1.y), bf2(v1.z, v1.w));
          }
          const uint32_t off = koff(row, c8 * 8, sbo1, 128);
          *reinterpret_cast<uint4*>(ah + off) = h;
          if (SPLIT) *reinterpret_cast<uint4*>(ah + p.a1_bytes + off) = l;
        }
        mbar_arrive(&empty[s]);
        fence_proxy_async();
        fence_before_sync();
        named_sync(1, 128);
        if (*sflag) ok = false;
        if (!ok) break;
        fence_after_sync();
        if (tid == 0) {
          const uint32_t d = tbase + (uint32_t)(j * p.N1);
          const uint32_t sa = smem_u32(ah), sb = smem_u32(b1);
          for (int ks = 0; ks < p.K1 / 16; ++ks) {
            const uint32_t ko = (uint32_t)ks * 256u;
            const uint64_t ahd = sdesc(sa + ko, 128, sbo1), bhd = sdesc(sb + ko, 128, sbo1);
            mma_bf16(d, ahd, bhd, idt, ks > 0 ? 1u : 0u);
            if (SPLIT) {
              mma_bf16(d, ahd, sdesc(sb + p.b1_bytes + ko, 128, sbo1), idt, 1u);
              mma_bf16(d, sdesc(sa + p.a1_bytes + ko, 128, sbo1), bhd, idt, 1u);
            }
          }
          mma_commit(&bar_t[bb]);
        }
        ++cnt_t[bb];
        ++it;
      }
      if (!ok) break;
      // all t-stage MMAs of the group are complete once the last commit lands
      {
        const int bl = (int)((it - 1) & 1);
        if (!mbar_wait(&bar_t[bl], (cnt_t[bl] - 1) & 1, kWaitCycles)) {
          atomicExch(p.err, 1);
          *sflag = 1;
        }
        named_sync(1, 128);
        if (*sflag) ok = false;
        if (!ok) break;
      }
      fence_after_sync();
      // ---- z stage: P^T from TMEM into the K-major A2 operand, hi pass then lo pass ----
      const int npass = SPLIT ? 2 : 1;
      for (int pass = 0; pass < npass; ++pass) {
        for (int j = 0; j < ntile; ++j) {
          uint32_t v[16];
          tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * p.N1), v);
          tmem_ld_wait();
          const int cl = j * p.cpt + r / Nz;  // column within the group
          const int z = r % Nz;
          if (cl < gcols) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              if (q >= 2 * Jt) break;
              const float x = __uint_as_float(v[q]);
              const __nv_bfloat16 h = __float2bfloat16_rn(x);
              const __nv_bfloat16 o = pass == 0 ? h : __float2bfloat16_rn(x - __bfloat162float(h));
              const int m = cl * Jt + (q >> 1);
              const int k = (q & 1) * Nz + z;
              *reinterpret_cast<__nv_bfloat16*>(a2 + koff(m, k, p.sbo2, p.lbo2)) = o;
            }
          }
        }
        fence_proxy_async();
        fence_before_sync();
        named_sync(1, 128);
        fence_after_sync();
        if (tid == 0) {
          const uint32_t d = tbase + p.d2_col;
          const uint32_t sa = smem_u32(a2), sb = smem_u32(b2);
          for (int ks = 0; ks < p.K2 / 16; ++ks) {
            const uint64_t ad = sdesc(sa + (uint32_t)ks * 2u * p.lbo2, p.lbo2, p.sbo2);
            const uint32_t kb = (uint32_t)ks * 256u;
            if (pass == 0) {
              mma_bf16(d, ad, sdesc(sb + kb, 128, sbo_b2), idz, ks > 0 ? 1u : 0u);
              if (SPLIT) mma_bf16(d, ad, sdesc(sb + p.b2_bytes + kb, 128, sbo_b2), idz, 1u);
            } else {
              mma_bf16(d, ad, sdesc(sb + kb, 128, sbo_b2), idz, 1u);
            }
          }
          mma_commit(&bar_z[0]);
        }
        if (!mbar_wait(&bar_z[0], cnt_z & 1, kWaitCycles)) {
          atomicExch(p.err, 1);
          *sflag = 1;
        }
        ++cnt_z;
        named_sync(1, 128);
        if (*sflag) ok = false;
        fence_after_sync();
        if (!ok) break;
      }
      if (!ok) break;
      // ---- D2 rows (col, jt) -> T1[col][jz][jt] ----
      {
        const int m = r;
        const int cl = m / Jt, jt = m - cl * Jt;
        const bool valid = cl < gcols && m < p.G * Jt;
        float2* dst = p.out + ((gcol0 + cl) * Jz) * Jt + jt;
        for (int c0 = 0; c0 < p.N2; c0 += 16) {
          uint32_t v[16];
          tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + p.d2_col + (uint32_t)c0, v);
          tmem_ld_wait();
          if (valid) {
#pragma unroll
            for (int q = 0; q < 16; q += 2) {
              const int jz = (c0 + q) >> 1;
              if (jz < Jz)
                dst[(long long)jz * Jt] = make_float2(__uint_as_float(v[q]), __uint_as_float(v[q + 1]));
            }
          }
        }
      }
      fence_before_sync();
      named_sync(1, 128);
      fence_after_sync();
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0) tmem_dealloc(tbase, p.tmem_cols);
}

static bool fwd_tz_plan(const Dims& d, FwdTcK& k, size_t& smem, char* why, size_t nwhy) {
  auto no = [&](const char* m) {
    if (why) snprintf(why, nwhy, "tensor-core t,z stage: %s", m);
    return false;
  };
  if (d.Nz < 8 || d.Nz > 128 || 128 % d.Nz != 0) return no("Nz must divide 128 (8..128)");
  if (d.Nt % 8 != 0 || d.Nt > 64) return no("Nt must be a multiple of 8, at most 64");
  if (2 * d.Jt > 16) return no("mt must be <= 8");
  if (2 * d.Jz > 128) return no("2*mz must be <= 64");
  k.Nz = (int)d.Nz;
  k.Nt = (int)d.Nt;
  k.Jz = (int)d.Jz;
  k.Jt = (int)d.Jt;
  k.cpt = (int)(128 / d.Nz);
  int G = (int)(128 / d.Jt);
  G = G / k.cpt * k.cpt;
  if (G < k.cpt) return no("mt too large for the column grouping");
  k.G = G;
  k.tpg = G / k.cpt;
  k.K1 = (int)up((uint32_t)d.Nt, 16);
  k.N1 = 16;
  k.K2 = (int)(2 * d.Nz);
  k.N2 = (int)up((uint32_t)(2 * d.Jz), 16);
  k.lbo2 = 144;
  k.sbo2 = (uint32_t)(k.K2 / 8) * k.lbo2;
  const uint32_t tcols = (uint32_t)(k.tpg * k.N1);
  k.d2_col = tcols;
  if (tcols + k.N2 > 512) return no("too many TMEM columns");
  k.tmem_cols = pow2_cols(tcols + (uint32_t)k.N2);
  k.xf_bytes = (uint32_t)(128 * d.Nt * 4);
  k.a1_bytes = (uint32_t)(128 * k.K1 * 2);
  k.b1_bytes = (uint32_t)(k.N1 * k.K1 * 2);
  k.b2_bytes = (uint32_t)(k.N2 * k.K2 * 2);
  const uint32_t a2_bytes = 16u * k.sbo2;
  // pick the deepest ring that fits
  for (int S = 6; S >= 2; --S) {
    uint32_t off = 0;
    k.o_xf = off;
    off += (uint32_t)S * k.xf_bytes;
    k.o_a1 = off = up(off, 1024);
    off += 4 * k.a1_bytes;
    k.o_b1 = off = up(off, 128);
    off += 2 * k.b1_bytes;
    k.o_a2 = off = up(off, 128);
    off += a2_bytes;
    k.o_b2 = off = up(off, 128);
    off += 2 * k.b2_bytes;
    k.o_bar = off = up(off, 16);
    off += (uint32_t)(2 * S + 3) * 8 + 16;
    if (off <= 227 * 1024) {
      k.S = S;
      // one CTA per SM when the TMEM allocation would not fit twice
      smem = (k.tmem_cols > 256 && off < 116 * 1024) ? 116 * 1024 : off;
      return true;
    }
  }
  return no("shared memory does not fit");
}

bool fwd_tz_tc_supported(const Dims& d, char* why, size_t nwhy) {
  FwdTcK k{};
  size_t smem = 0;
  return fwd_tz_plan(d, k, smem, why, nwhy);
}

cudaError_t launch_fwd_tz_tc(const float* in, float2* out, int64_t ncol, const Dims& d,
                             const float2* ft, const float2* fz, bool split, int* err,
                             cudaStream_t s) {
  if (ncol <= 0) return cudaSuccess;
  FwdTcK k{};
  size_t smem = 0;
  if (!fwd_tz_plan(d, k, smem, nullptr, 0)) return cudaErrorInvalidValue;
  k.in = in;
  k.out = out;
  k.Ft = ft;
  k.Fz = fz;
  k.err = err;
  k.ncol = ncol;
  k.ngroups = (ncol + k.G - 1) / k.G;
  const void* kern = split ? (const void*)k_fwd_tz_tc<true> : (const void*)k_fwd_tz_tc<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<long long>(k.ngroups, sm_count());
  if (split)
    FNO_LAUNCH_TC("fno_fwd_tz_tc_bf16x3", k_fwd_tz_tc<true>, grid, 160, smem, s, k);
  else
    FNO_LAUNCH_TC("fno_fwd_tz_tc_bf16", k_fwd_tz_tc<false>, grid, 160, smem, s, k);
  return cudaSuccess;
}

// ============================================================================
// Inverse z, t stages + epilogue
// ============================================================================
struct EpiTcK {
  const float2* U;
  const float* lin;
  const float* wlin;
  const float* bias;
  const float* dz;
  float* out;
  float* part;
  const float2* Iz;  // [Nz][Jz]
  const float2* It;  // [Jt][Nt]
  int* err;
  long long NxNy, ntiles;
  int Nz, Nt, Jz, Jt, Cs, Cl, w_si, w_sc;
  int zc, P, PS, nzc, NP, KX, KS, S;
  uint32_t o_xf, xf_bytes, o_ax, ax_bytes, o_bx, bx_bytes, o_as, as_bytes, o_bs, bs_bytes;
  uint32_t o_u, o_iz, o_bias, o_da, o_bar;
  uint32_t tmem_cols;
  int nblk, OB, KG;  // dW_lin blocking (EPI_DA)
};

template <int MODE, bool SPLIT>
__global__ void __launch_bounds__(256, 2) k_epi_tc(const EpiTcK p) {
  constexpr bool LIN = MODE != EPI_SPECTRAL;
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* xf = reinterpret_cast<float*>(sm + p.o_xf);
  unsigned char* ax = sm + p.o_ax;
  unsigned char* bx = sm + p.o_bx;
  unsigned char* as_ = sm + p.o_as;
  unsigned char* bs = sm + p.o_bs;
  float2* su = reinterpret_cast<float2*>(sm + p.o_u);
  float2* siz = reinterpret_cast<float2*>(sm + p.o_iz);
  float* sbias = reinterpret_cast<float*>(sm + p.o_bias);
  float* sda = reinterpret_cast<float*>(sm + p.o_da);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + p.o_bar);  // [S]
  uint64_t* bar_m = full + p.S;                                // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar_m + 2);
  int* sflag = reinterpret_cast<int*>(tslot + 1);
  const int S = p.S, Nz = p.Nz, Nt = p.Nt, Jz = p.Jz, Jt = p.Jt, Cs = p.Cs, Cl = p.Cl;
  const int P = p.P, PS = p.PS, NP = p.NP, KX = p.KX, KS = p.KS;
  const uint32_t sbo_x = (uint32_t)KX * 16u, sbo_s = (uint32_t)KS * 16u;
  const uint32_t band_bytes = (uint32_t)NP * (uint32_t)KS * 2u;
  const long long chan = p.NxNy * (long long)Nz * Nt;

  const long long t_begin = p.ntiles * blockIdx.x / gridDim.x;
  const long long t_end = p.ntiles * (blockIdx.x + 1) / gridDim.x;
  const int nloc = (int)(t_end - t_begin);

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
    mbar_init(&bar_m[0], 1);
    mbar_init(&bar_m[1], 1);
    *sflag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, p.tmem_cols);
    tmem_relinquish();
  }
  // constant operands and zero padding
  for (uint32_t e = tid; e < 2u * p.ax_bytes / 16u; e += 256) reinterpret_cast<uint4*>(ax)[e] = make_uint4(0, 0, 0, 0);
  for (uint32_t e = tid; e < 2u * p.bs_bytes / 16u; e += 256) reinterpret_cast<uint4*>(bs)[e] = make_uint4(0, 0, 0, 0);
  if (LIN) {
    for (int e = tid; e < NP * KX; e += 256) {
      const int o = e / KX, i = e - o * KX;
      const float v = (o < Cs && i < Cl) ? p.wlin[(long long)i * p.w_si + (long long)o * p.w_sc] : 0.f;
      __nv_bfloat16 h, l;
      split1(v, h, l);
      const uint32_t off = koff(o, i, sbo_x, 128);
      *reinterpret_cast<__nv_bfloat16*>(bx + off) = h;
      *reinterpret_cast<__nv_bfloat16*>(bx + p.bx_bytes + off) = l;
    }
  }
  {
    const int rows = 256 - Nt, r0 = 128 - Nt;
    for (int e = tid; e < rows * KS; e += 256) {
      const int r = e / KS, k = e - r * KS;
      const int t = r - r0;
      float v = 0.f;
      if (t >= 0 && t < Nt && k < 2 * Jt) {
        const float2 f = p.It[(k >> 1) * Nt + t];
        v = (k & 1) ? -f.y : f.x;
      }
      __nv_bfloat16 h, l;
      split1(v, h, l);
      const uint32_t off = koff(r, k, sbo_s, 128);
      *reinterpret_cast<__nv_bfloat16*>(as_ + off) = h;
      *reinterpret_cast<__nv_bfloat16*>(as_ + p.as_bytes + off) = l;
    }
  }
  if (MODE == EPI_FWD || MODE == EPI_DA)
    for (int c = tid; c < Cs; c += 256) sbias[c] = p.bias[c];
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t idv = idesc(kFmtBF16, 128, NP);

  auto issue = [&](long long tau, int s) {
    const long long col = tau / p.nzc;
    const int z0 = (int)(tau - col * p.nzc) * p.zc;
    const int zn = min(p.zc, Nz - z0);
    const long long b = col / p.NxNy, xy = col - b * p.NxNy;
    const uint32_t bytes = (uint32_t)(zn * Nt * 4);
    mbar_arrive_expect_tx(&full[s], bytes * (uint32_t)Cl);
    for (int i = 0; i < Cl; ++i) {
      const float* src = p.lin + (b * Cl + i) * chan + xy * (long long)(Nz * Nt) + (long long)z0 * Nt;
      bulk_g2s(xf + ((size_t)s * Cl + i) * PS, src, bytes, &full[s]);
    }
  };
  int issued = 0;
  if (LIN && tid == 0)
    for (; issued < S && issued < nloc; ++issued) issue(t_begin + issued, issued);

  // dW_lin accumulators (EPI_DA): thread -> (i block, o block, point group)
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;

  long long cur_col = -1;
  bool ok = true;
  int consumed = 0;
  for (int n = 0; n <= nloc; ++n) {
    const bool have = n < nloc;
    if (have) {
      const long long tau = t_begin + n;
      const long long col = tau / p.nzc;
      const int z0 = (int)(tau - col * p.nzc) * p.zc;
      const int zn = min(p.zc, Nz - z0);
      const long long b = col / p.NxNy, xy = col - b * p.NxNy;
      if (col != cur_col) {
        __syncthreads();
        const int JZT = Jz * Jt;
        for (int e = tid; e < Cs * JZT; e += 256) {
          const int c = e / JZT, q = e - c * JZT;
          su[e] = p.U[((b * Cs + c) * p.NxNy + xy) * JZT + q];
        }
        cur_col = col;
      }
      for (int e = tid; e < zn * Jz; e += 256) siz[e] = p.Iz[z0 * Jz + e];
      bool w_ok = true;
      if (LIN) w_ok = mbar_wait(&full[n % S], (uint32_t)((n / S) & 1), kWaitCycles);
      if (n >= 1) w_ok = w_ok && mbar_wait(&bar_m[(n - 1) & 1], (uint32_t)(((n - 1) >> 1) & 1), kWaitCycles);
      if (!w_ok) *sflag = 1;
      if (LIN && w_ok) consumed = n + 1;
      __syncthreads();  // su, siz visible; MMA(n-1) done
      fence_after_sync();
      if (*sflag) {
        ok = false;
      } else {
        // A_X: rows p (points), K = lin channels, from the fp32 staging [Cl][PS]
        if (LIN) {
          const float* xs = xf + (size_t)(n % S) * Cl * PS;
          const int ich = (Cl + 7) / 8;
          const int valid = zn * Nt;
          for (int e = tid; e < P * ich; e += 256) {
            const int pt = e % P, ic = e / P;
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int i = ic * 8 + j;
              v[j] = (i < Cl && pt < valid) ? xs[i * PS + pt] : 0.f;
            }
            uint4 h, l;
            if (SPLIT) {
              split2(v[0], v[1], h.x, l.x);
              split2(v[2], v[3], h.y, l.y);
              split2(v[4], v[5], h.z, l.z);
              split2(v[6], v[7], h.w, l.w);
            } else {
              h = make_uint4(bf2(v[0], v[1]), bf2(v[2], v[3]), bf2(v[4], v[5]), bf2(v[6], v[7]));
            }
            const uint32_t off = koff(pt, ic * 8, sbo_x, 128);
            *reinterpret_cast<uint4*>(ax + off) = h;
            if (SPLIT) *reinterpret_cast<uint4*>(ax + p.ax_bytes + off) = l;
          }
        }
        // B_S: Q[c][zz][jt] = sum_jz Iz[z][jz] U[c][jz][jt], one band per z plane
        {
          const int JZT = Jz * Jt;
          for (int e = tid; e < Cs * zn * Jt; e += 256) {
            const int jt = e % Jt;
            const int zz = (e / Jt) % zn;
            const int c = e / (Jt * zn);
            const float2* u = su + c * JZT + jt;
            const float2* iz = siz + zz * Jz;
            float re = 0.f, im = 0.f;
            for (int jz = 0; jz < Jz; ++jz) {
              const float2 f = iz[jz], v = u[jz * Jt];
              re = fmaf(f.x, v.x, re);
              re = fmaf(-f.y, v.y, re);
              im = fmaf(f.x, v.y, im);
              im = fmaf(f.y, v.x, im);
            }
            const uint32_t off = (uint32_t)zz * band_bytes + koff(c, 2 * jt, sbo_s, 128);
            if (SPLIT) {
              uint32_t h, l;
              split2(re, im, h, l);
              *reinterpret_cast<uint32_t*>(bs + off) = h;
              *reinterpret_cast<uint32_t*>(bs + p.bs_bytes + off) = l;
            } else {
              *reinterpret_cast<uint32_t*>(bs + off) = bf2(re, im);
            }
          }
        }
        fence_proxy_async();
        fence_before_sync();
      }
      __syncthreads();
      if (*sflag) ok = false;
      if (!ok) break;
      fence_after_sync();
      if (tid == 0) {
        const uint32_t d = tbase + (uint32_t)((n & 1) * NP);
        uint32_t accf = 0;
        if (LIN) {
          const uint32_t sa = smem_u32(ax), sb = smem_u32(bx);
          for (int ks = 0; ks < KX / 16; ++ks) {
            const uint32_t ko = (uint32_t)ks * 256u;
            const uint64_t ah = sdesc(sa + ko, 128, sbo_x), bh = sdesc(sb + ko, 128, sbo_x);
            mma_bf16(d, ah, bh, idv, accf);
            accf = 1;
            if (SPLIT) {
              mma_bf16(d, ah, sdesc(sb + p.bx_bytes + ko, 128, sbo_x), idv, 1u);
              mma_bf16(d, sdesc(sa + p.ax_bytes + ko, 128, sbo_x), bh, idv, 1u);
            }
          }
        }
        const uint32_t sa = smem_u32(as_), sb = smem_u32(bs);
        for (int zz = 0; zz < zn; ++zz) {
          const uint32_t start_row = (uint32_t)(128 - Nt - zz * Nt);
          const uint32_t ao = (start_row >> 3) * sbo_s;
          const uint32_t bo = (uint32_t)zz * band_bytes;
          for (int ks = 0; ks < KS / 16; ++ks) {
            const uint32_t ko = (uint32_t)ks * 256u;
            const uint64_t ah = sdesc(sa + ao + ko, 128, sbo_s), bh = sdesc(sb + bo + ko, 128, sbo_s);
            mma_bf16(d, ah, bh, idv, accf);
            accf = 1;
            if (SPLIT) {
              mma_bf16(d, ah, sdesc(sb + p.bs_bytes + bo + ko, 128, sbo_s), idv, 1u);
              mma_bf16(d, sdesc(sa + p.as_bytes + ao + ko, 128, sbo_s), bh, idv, 1u);
            }
          }
        }
        mma_commit(&bar_m[n & 1]);
      }
    } else if (n >= 1) {
      if (!mbar_wait(&bar_m[(n - 1) & 1], (uint32_t)(((n - 1) >> 1) & 1), kWaitCycles)) *sflag = 1;
      __syncthreads();
      if (*sflag) {
        ok = false;
        break;
      }
      fence_after_sync();
    }
    // ---- epilogue of tile n-1 ----
    if (n >= 1) {
      const long long tau = t_begin + n - 1;
      const long long col = tau / p.nzc;
      const int z0 = (int)(tau - col * p.nzc) * p.zc;
      const int zn = min(p.zc, Nz - z0);
      const long long b = col / p.NxNy, xy = col - b * p.NxNy;
      const int valid = zn * Nt;
      const int q = warp & 3, half = warp >> 2;
      const int row = q * 32 + lane;
      const long long pofs = xy * (long long)(Nz * Nt) + (long long)z0 * Nt + row;
      const uint32_t ta = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(((n - 1) & 1) * NP + half * (NP / 2));
      for (int c0 = 0; c0 < NP / 2; c0 += 8) {
        uint32_t v[8];
        tmem_ld8(ta + (uint32_t)c0, v);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int o = half * (NP / 2) + c0 + j;
          if (o < Cs && row < valid) {
            const float a = __uint_as_float(v[j]);
            const long long oofs = (b * Cs + o) * chan + pofs;
            if (MODE == EPI_FWD) {
              p.out[oofs] = gelu_f(a + sbias[o]);
            } else if (MODE == EPI_DA) {
              const float da = p.dz[oofs] * gelu_grad_f(a + sbias[o]);
              p.out[oofs] = da;
              sda[o * (P + 1) + row] = da;
            } else {
              p.out[oofs] = a;
            }
          }
        }
      }
      fence_before_sync();
      if (MODE == EPI_DA) {
        // dW_lin[i][o] += sum_p x[i][p] dA[o][p]; channel i == Cl is the ones row (db)
        __syncthreads();
        const float* xs = xf + (size_t)((n - 1) % S) * Cl * PS;
        if (tid < p.nblk * p.KG) {
          const int blk = tid % p.nblk, kg = tid / p.nblk;
          const int i0 = (blk / p.OB) * 4, o0 = (blk % p.OB) * 4;
          const int pa = kg * P / p.KG, pb = min((kg + 1) * P / p.KG, valid);
          for (int pt = pa; pt < pb; ++pt) {
            float xv[4], dv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
              const int i = i0 + a;
              xv[a] = i < Cl ? xs[i * PS + pt] : (i == Cl ? 1.f : 0.f);
              const int o = o0 + a;
              dv[a] = o < Cs ? sda[o * (P + 1) + pt] : 0.f;
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(xv[a], dv[c], acc[a][c]);
          }
        }
      }
    }
    // release the staging of tile n-1 and refill it
    if (LIN && n >= 1) {
      __syncthreads();
      if (tid == 0 && issued < nloc && issued == n - 1 + S) {
        issue(t_begin + issued, (n - 1) % S);
        ++issued;
      }
    }
  }
  if (!ok) atomicExch(p.err, 1);
  // drain copies that were issued but not consumed (error path)
  if (LIN && tid == 0)
    for (int k = consumed; k < issued; ++k) mbar_wait(&full[k % S], (uint32_t)((k / S) & 1), kWaitCycles);
  __syncthreads();
  if (MODE == EPI_DA) {
    // fixed-order reduction of the per-thread partial sums over point groups
    float* red = xf;  // the staging ring is free now
    const int nacc = p.nblk * p.KG;
    if (tid < nacc) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) red[tid * 16 + a * 4 + c] = acc[a][c];
    }
    __syncthreads();
    const int npair = Cl * Cs + Cs;
    for (int e = tid; e < p.nblk * 16; e += 256) {
      const int blk = e / 16, a = (e / 4) % 4, c = e % 4;
      const int i = (blk / p.OB) * 4 + a, o = (blk % p.OB) * 4 + c;
      float sum = 0.f;
      for (int kg = 0; kg < p.KG; ++kg) sum += red[(kg * p.nblk + blk) * 16 + a * 4 + c];
      if (o < Cs && i <= Cl) {
        const int idx = (i < Cl) ? i * Cs + o : Cl * Cs + o;
        p.part[(long long)blockIdx.x * npair + idx] = sum;
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0) tmem_dealloc(tbase, p.tmem_cols);
}

int epilogue_tc_max_grid() { return 1024; }

static bool epi_plan(const Dims& d, int mode, int Cs, int Cl, EpiTcK& k, size_t& smem,
                     int& per_sm, char* why, size_t nwhy) {
  auto no = [&](const char* m) {
    if (why) snprintf(why, nwhy, "tensor-core epilogue: %s", m);
    return false;
  };
  if (d.Nt % 8 != 0 || d.Nt > 128 || 128 % d.Nt != 0) return no("Nt must divide 128 and be a multiple of 8");
  if (2 * d.Jt > 32) return no("mt must be <= 16");
  if (Cs > 64 || (mode != EPI_SPECTRAL && Cl > 64)) return no("channels must be <= 64");
  k.Nz = (int)d.Nz;
  k.Nt = (int)d.Nt;
  k.Jz = (int)d.Jz;
  k.Jt = (int)d.Jt;
  k.Cs = Cs;
  k.Cl = mode == EPI_SPECTRAL ? 0 : Cl;
  k.zc = (int)std::min<int64_t>(d.Nz, 128 / d.Nt);
  k.P = k.zc * (int)d.Nt;
  k.PS = k.P + 4;
  k.nzc = (int)((d.Nz + k.zc - 1) / k.zc);
  k.NP = (int)up((uint32_t)Cs, 16);
  k.KX = k.Cl > 0 ? (int)up((uint32_t)k.Cl, 16) : 0;
  k.KS = (int)up((uint32_t)(2 * d.Jt), 16);
  k.tmem_cols = pow2_cols(2u * (uint32_t)k.NP);
  k.ax_bytes = (uint32_t)(128 * std::max(k.KX, 16) * 2);
  k.bx_bytes = (uint32_t)(k.NP * std::max(k.KX, 16) * 2);
  k.as_bytes = (uint32_t)((256 - d.Nt) * k.KS * 2);
  k.bs_bytes = (uint32_t)(k.zc * k.NP * k.KS * 2);
  if (mode == EPI_DA) {
    const int IB = (k.Cl + 1 + 3) / 4;
    k.OB = (Cs + 3) / 4;
    k.nblk = IB * k.OB;
    k.KG = std::max(1, std::min(256 / k.nblk, k.P));
  } else {
    k.OB = k.nblk = k.KG = 1;
  }
  for (int want = 2; want >= 1; --want) {
    for (int S = 4; S >= 2; --S) {
      uint32_t off = 0;
      k.xf_bytes = (uint32_t)(std::max(k.Cl, 1) * k.PS * 4);
      k.o_xf = off;
      uint32_t xf_total = (uint32_t)S * k.xf_bytes;
      if (mode == EPI_DA) xf_total = std::max(xf_total, (uint32_t)(k.nblk * k.KG * 16 * 4));
      off += xf_total;
      k.o_ax = off = up(off, 128);
      off += 2 * k.ax_bytes;
      k.o_bx = off = up(off, 128);
      off += 2 * k.bx_bytes;
      k.o_as = off = up(off, 128);
      off += 2 * k.as_bytes;
      k.o_bs = off = up(off, 128);
      off += 2 * k.bs_bytes;
      k.o_u = off = up(off, 16);
      off += (uint32_t)(Cs * d.Jz * d.Jt * 8);
      k.o_iz = off = up(off, 16);
      off += (uint32_t)(k.zc * d.Jz * 8);
      k.o_bias = off = up(off, 16);
      off += (uint32_t)(Cs * 4);
      k.o_da = off = up(off, 16);
      if (mode == EPI_DA) off += (uint32_t)(Cs * (k.P + 1) * 4);
      k.o_bar = off = up(off, 16);
      off += (uint32_t)(S + 2) * 8 + 16;
      const uint32_t limit = want == 2 ? 113 * 1024 : 227 * 1024;
      if (off <= limit && (uint32_t)want * k.tmem_cols <= 512) {
        k.S = S;
        smem = off;
        per_sm = want;
        return true;
      }
    }
  }
  return no("shared memory does not fit");
}

bool epilogue_tc_supported(const Dims& d, int mode, int Cs, int Cl, char* why, size_t nwhy) {
  EpiTcK k{};
  size_t smem = 0;
  int per_sm = 0;
  return epi_plan(d, mode, Cs, Cl, k, smem, per_sm, why, nwhy);
}

template <int MODE, bool SPLIT>
static cudaError_t launch_epi_tc_t(const EpiTcK& k, size_t smem, int grid, cudaStream_t s) {
  const void* kern = (const void*)k_epi_tc<MODE, SPLIT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  static const char* names[2][4] = {
      {"fno_epi_spectral_tc_bf16", "fno_epi_fwd_tc_bf16", "fno_epi_da_tc_bf16", "fno_epi_dx_tc_bf16"},
      {"fno_epi_spectral_tc_bf16x3", "fno_epi_fwd_tc_bf16x3", "fno_epi_da_tc_bf16x3",
       "fno_epi_dx_tc_bf16x3"}};
  FNO_LAUNCH_TC(names[SPLIT ? 1 : 0][MODE], (k_epi_tc<MODE, SPLIT>), grid, 256, smem, s, k);
  return cudaSuccess;
}

cudaError_t launch_epilogue_tc(const Dims& d, const EpiArgs& a, bool split, int* err,
                               int* grid_used, cudaStream_t s) {
  if (d.B <= 0) {
    if (grid_used) *grid_used = 0;
    return cudaSuccess;
  }
  EpiTcK k{};
  size_t smem = 0;
  int per_sm = 1;
  if (!epi_plan(d, a.mode, a.Cs, a.Cl, k, smem, per_sm, nullptr, 0)) return cudaErrorInvalidValue;
  k.U = a.U;
  k.lin = a.lin_in;
  k.wlin = a.wlin;
  k.bias = a.bias;
  k.dz = a.dz;
  k.out = a.out;
  k.part = a.part;
  k.Iz = a.Iz;
  k.It = a.It;
  k.err = err;
  k.w_si = a.w_si;
  k.w_sc = a.w_sc;
  k.NxNy = d.Nx * d.Ny;
  k.ntiles = d.B * d.Nx * d.Ny * (long long)k.nzc;
  int grid = (int)std::min<long long>(k.ntiles, (long long)per_sm * sm_count());
  grid = std::min(grid, epilogue_tc_max_grid());
  if (grid_used) *grid_used = grid;
  switch (a.mode) {
    case EPI_SPECTRAL:
      return split ? launch_epi_tc_t<EPI_SPECTRAL, true>(k, smem, grid, s)
                   : launch_epi_tc_t<EPI_SPECTRAL, false>(k, smem, grid, s);
    case EPI_FWD:
      return split ? launch_epi_tc_t<EPI_FWD, true>(k, smem, grid, s)
                   : launch_epi_tc_t<EPI_FWD, false>(k, smem, grid, s);
    case EPI_DA:
      return split ? launch_epi_tc_t<EPI_DA, true>(k, smem, grid, s)
                   : launch_epi_tc_t<EPI_DA, false>(k, smem, grid, s);
    default:
      return split ? launch_epi_tc_t<EPI_DX, true>(k, smem, grid, s)
                   : launch_epi_tc_t<EPI_DX, false>(k, smem, grid, s);
  }
}

}  // namespace fno
