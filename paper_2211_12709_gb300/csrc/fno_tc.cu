// fno_tc.cu -- tensor-core kernel of the forward pruned DFT over t then z of
// every (b, c, x, y) column: the first half of F_yzt, S_yzt in Alg. 2 of the
// paper, which carries a full read of the block input.
//
//   t stage  P[(col,z)][(ri,jt)] = X[(col,z)][t] . Ft[(ri,jt)][t]   (mma.sync)
//   z stage  D2[(col,ri,jt)][(jz,f)] = P_ri[col][z][jt] . F_f[jz][z] (tcgen05)
//
// Input tiles arrive by bulk copy (TMA engine) into a ring.  The t stage is a
// skinny GEMM (N = 16): one tcgen05.mma with M = 128, K = 16 was measured at
// about 153 SM cycles whatever N, so there it runs as warp-level mma.sync
// (about 965 MAC/clk/SM) straight from the ring into the MN-major z-stage
// operand; the z stage (K = Nz, every column of a group in M) stays on tcgen05
// with its accumulator in TMEM.  Precision: BF16 operands (one product) or
// split BF16 (x = hi + lo, products hi.hi + hi.lo + lo.hi), FP32 accumulation.
// Every wait is bounded; on timeout the kernel raises *err, drains what it
// started and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>

#include "fno_internal.h"
#include "umma.h"

namespace fno {

using namespace umma;


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
// Round to TF32 (10 stored mantissa bits, nearest, ties away); a TF32 value is
// exact as BF16 hi + lo, so the split products reproduce TF32 arithmetic.
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t y;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
  return __uint_as_float(y);
}
template <bool TF>
__device__ __forceinline__ float rnd(float x) {
  return TF ? tf32_round(x) : x;
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
// Warp roles (448 threads): warp 0 producer (bulk copies of 128-row tiles into a
// ring), warp 1 tcgen05 issuer of the z stage, warps 2-9 t stage (mma.sync from
// the ring straight into the MN-major z-stage operand, one 16-row m-tile each),
// warps 10-13 readback (D2 in TMEM -> T1 in global memory).  Roles hand work to each other through
// mbarriers only; the z-stage operand and D2 are double-buffered per group.
//
// t stage of a 16-row m-tile (rows = (column, z), n = (ri, jt), k = t):
//   P[row][(ri, jt)] = sum_t X[row][t] Ft_ri[jt][t]     (mma.sync m16n8k16)
//   the k slots of a thread map to 4 consecutive t (one float4 of the row), and
//   the B fragments of the basis use the same map.
// z-stage GEMM of a group of kG = 8 columns (tcgen05, M = 128):
//   rows m = col * 16 + ri * 8 + jt   (P_re rows, then P_im rows, jt padded to 8)
//   cols n = 2 * jz + f                (f = 0: cos rows of Fz, f = 1: -sin rows)
//   D2[m][n] = sum_z P_ri[col][z][jt] * F_f[jz][z]
//   T_re = D2[(col,0,jt)][(jz,0)] - D2[(col,1,jt)][(jz,1)]
//   T_im = D2[(col,1,jt)][(jz,0)] + D2[(col,0,jt)][(jz,1)]
constexpr int kG = 8;
constexpr int kFwdThreads = 448;
constexpr int kTWarps = 8;  // t-stage warps
constexpr int kTThreads = 32 * kTWarps;
constexpr int kKSMax = 4;  // t-stage k-steps of 16 (Nt <= 64)

struct FwdTcK {
  const float* in;
  float2* out;
  const float2* Ft;  // [Jt][Nt]  (cos, -sin) * scale
  const float2* Fz;  // [Jz][Nz]  (cos, -sin)
  int* err;
  long long ncol, ngroups;
  int Nz, Nt, Jz, Jt, cpt, tpg, KS, N2, S;
  uint32_t o_xf, xf_bytes, o_a2, a2_bytes, o_b2, b2_bytes, o_bar;
  uint32_t tmem_cols;
  uint32_t a2_stride;  // bytes between the two z-operand buffers (hi and, when split, lo)
};

__device__ __forceinline__ void mma_sync16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                           uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <bool SPLIT, bool TF>
__global__ void __launch_bounds__(kFwdThreads, 1) k_fwd_tz_tc(const FwdTcK p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* xf = sm + p.o_xf;
  unsigned char* a2 = sm + p.o_a2;  // buffer b: hi at a2 + b * a2_stride, lo (split) after it
  unsigned char* b2 = sm + p.o_b2;
  const int S = p.S;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + p.o_bar);
  uint64_t* empty = full + S;
  uint64_t* a2full = empty + S;   // [2] t stage -> z-stage issuer (kTThreads arrivals)
  uint64_t* zdone = a2full + 2;   // [2] z-stage MMAs of a buffer complete (commit)
  uint64_t* d2empty = zdone + 2;  // [2] readback of a D2 buffer done (128 arrivals)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(d2empty + 2);
  volatile int* sflag = reinterpret_cast<volatile int*>(tslot + 1);
  const int Nz = p.Nz, Nt = p.Nt, Jz = p.Jz, Jt = p.Jt;
  const uint32_t sbo_b2 = (uint32_t)Nz * 16u;
  const uint32_t kg_a2 = 2048u;  // MN-major: K group stride (16 row groups of 128 B)

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kTThreads);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&a2full[b], kTThreads);
      mbar_init(&zdone[b], 1);
      mbar_init(&d2empty[b], 128);
    }
    *sflag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tslot, p.tmem_cols);
    tmem_relinquish();
  }
  for (uint32_t e = tid; e < p.a2_stride * 2u / 16u; e += kFwdThreads)
    reinterpret_cast<uint4*>(a2)[e] = make_uint4(0, 0, 0, 0);
  for (int e = tid; e < p.N2 * Nz; e += kFwdThreads) {
    const int n = e / Nz, z = e - n * Nz;
    float v = 0.f;
    if (n < 2 * Jz) {
      const float2 f = p.Fz[(n >> 1) * Nz + z];
      v = (n & 1) ? f.y : f.x;
    }
    __nv_bfloat16 h, l;
    split1(rnd<TF>(v), h, l);
    const uint32_t off = koff(n, z, sbo_b2, 128);
    *reinterpret_cast<__nv_bfloat16*>(b2 + off) = h;
    *reinterpret_cast<__nv_bfloat16*>(b2 + p.b2_bytes + off) = l;
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = *tslot;

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      long long it = 0;
      bool ok = true;
      for (long long g = blockIdx.x; g < p.ngroups && ok; g += gridDim.x) {
        const long long col0 = g * kG;
        const int gcols = (int)min((long long)kG, p.ncol - col0);
        const int ntile = (gcols + p.cpt - 1) / p.cpt;
        for (int j = 0; j < ntile; ++j) {
          const long long tc0 = col0 + (long long)j * p.cpt;
          const uint32_t bytes = (uint32_t)(min((long long)p.cpt, p.ncol - tc0) * Nz * Nt * 4);
          const int s = (int)(it % S);
          if (!mbar_wait(&empty[s], (uint32_t)(((it / S) & 1) ^ 1), kWaitCycles) || *sflag) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[s], bytes);
          bulk_g2s(xf + (size_t)s * p.xf_bytes, p.in + tc0 * Nz * Nt, bytes, &full[s]);
          ++it;
        }
      }
      if (!ok) {
        atomicExch(p.err, 1);
        *sflag = 1;
      }
      for (long long k = (it > S ? it - S : 0); k < it; ++k)
        mbar_wait(&full[k % S], (uint32_t)((k / S) & 1), kWaitCycles);
    }
  } else if (warp == 1) {
    // ---------------- z-stage issuer (tcgen05) ----------------
    if (lane == 0) {
      const uint32_t idz = idesc(kFmtBF16, 128, p.N2) | (1u << 15);  // A2 is MN-major
      long long gl = 0;
      bool ok = true;
      for (long long g = blockIdx.x; g < p.ngroups; g += gridDim.x, ++gl) {
        const int gb = (int)(gl & 1);
        if (!mbar_wait(&a2full[gb], (uint32_t)((gl >> 1) & 1), kWaitCycles) ||
            !mbar_wait(&d2empty[gb], (uint32_t)(((gl >> 1) & 1) ^ 1), kWaitCycles) || *sflag) {
          ok = false;
          break;
        }
        fence_after_sync();
        const uint32_t d = tbase + (uint32_t)gb * (uint32_t)p.N2;
        const uint32_t sa = smem_u32(a2 + (size_t)gb * p.a2_stride), sb = smem_u32(b2);
        for (int ks = 0; ks < Nz / 16; ++ks) {
          const uint64_t ah = sdesc(sa + (uint32_t)ks * 2u * kg_a2, kg_a2, 128);
          const uint64_t bh = sdesc(sb + (uint32_t)ks * 256u, 128, sbo_b2);
          mma_bf16(d, ah, bh, idz, ks > 0 ? 1u : 0u);
          if (SPLIT) {
            mma_bf16(d, ah, sdesc(sb + p.b2_bytes + (uint32_t)ks * 256u, 128, sbo_b2), idz, 1u);
            mma_bf16(d, sdesc(sa + p.a2_bytes + (uint32_t)ks * 2u * kg_a2, kg_a2, 128), bh, idz, 1u);
          }
        }
        mma_commit(&zdone[gb]);
      }
      if (!ok) {
        atomicExch(p.err, 1);
        *sflag = 1;
      }
      // every issued MMA must be complete before TMEM is released
      if (gl >= 1) mbar_wait(&zdone[(gl - 1) & 1], (uint32_t)(((gl - 1) >> 1) & 1), kWaitCycles);
    }
  } else if (warp < 2 + kTWarps) {
    // ---------------- t stage (mma.sync) ----------------
    const int tw = warp - 2;  // m-tile tw (rows 16 tw .. 16 tw + 15) of each 128-row tile
    const int g8 = lane >> 2, t4 = lane & 3;
    // basis B fragments: k slots 2 t4 + {0,1} <-> t = 16 ks + 4 t4 + {0,1},
    // slots 2 t4 + 8 + {0,1} <-> t = 16 ks + 4 t4 + {2,3}; n = jt = g8
    uint32_t bfh[2][kKSMax][2], bfl[2][kKSMax][2];
#pragma unroll
    for (int ri = 0; ri < 2; ++ri)
#pragma unroll
      for (int ks = 0; ks < kKSMax; ++ks) {
        auto F = [&](int t) -> float {
          if (g8 >= Jt || t >= Nt) return 0.f;
          const float2 f = p.Ft[g8 * Nt + t];
          return rnd<TF>(ri ? f.y : f.x);
        };
        const int t0 = 16 * ks + 4 * t4;
        split2(F(t0), F(t0 + 1), bfh[ri][ks][0], bfl[ri][ks][0]);
        split2(F(t0 + 2), F(t0 + 3), bfh[ri][ks][1], bfl[ri][ks][1]);
      }
    long long it = 0, gl = 0;
    bool ok = true;
    for (long long g = blockIdx.x; g < p.ngroups && ok; g += gridDim.x, ++gl) {
      const int gb = (int)(gl & 1);
      const long long col0 = g * kG;
      const int gcols = (int)min((long long)kG, p.ncol - col0);
      const int ntile = (gcols + p.cpt - 1) / p.cpt;
      // the z stage of group gl - 2 has finished reading this operand buffer
      if (gl >= 2 && !mbar_wait(&zdone[gb], (uint32_t)(((gl - 2) >> 1) & 1), kWaitCycles)) {
        ok = false;
        break;
      }
      unsigned char* ah2 = a2 + (size_t)gb * p.a2_stride;
      for (int j = 0; j < ntile; ++j) {
        const int s = (int)(it % S);
        const long long tc0 = col0 + (long long)j * p.cpt;
        const int rows = (int)min((long long)p.cpt, p.ncol - tc0) * Nz;
        if (!mbar_wait(&full[s], (uint32_t)((it / S) & 1), kWaitCycles) || *sflag) {
          ok = false;
          break;
        }
        const float* xs = reinterpret_cast<const float*>(xf + (size_t)s * p.xf_bytes);
        {
          const int r0 = 16 * tw + g8, r1 = r0 + 8;
          float acc[2][4];
#pragma unroll
          for (int ri = 0; ri < 2; ++ri)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[ri][q] = 0.f;
#pragma unroll
          for (int ks = 0; ks < kKSMax; ++ks) {
            if (ks < p.KS) {
              const int tt = 16 * ks + 4 * t4;
              float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
              if (tt < Nt) {
                if (r0 < rows) v0 = *reinterpret_cast<const float4*>(xs + r0 * Nt + tt);
                if (r1 < rows) v1 = *reinterpret_cast<const float4*>(xs + r1 * Nt + tt);
              }
              uint32_t ah[4], al[4];
              split2(rnd<TF>(v0.x), rnd<TF>(v0.y), ah[0], al[0]);
              split2(rnd<TF>(v1.x), rnd<TF>(v1.y), ah[1], al[1]);
              split2(rnd<TF>(v0.z), rnd<TF>(v0.w), ah[2], al[2]);
              split2(rnd<TF>(v1.z), rnd<TF>(v1.w), ah[3], al[3]);
              if (SPLIT) {
#pragma unroll
                for (int ri = 0; ri < 2; ++ri)
                  mma_sync16(acc[ri], al[0], al[1], al[2], al[3], bfh[ri][ks][0], bfh[ri][ks][1]);
#pragma unroll
                for (int ri = 0; ri < 2; ++ri)
                  mma_sync16(acc[ri], ah[0], ah[1], ah[2], ah[3], bfl[ri][ks][0], bfl[ri][ks][1]);
              }
#pragma unroll
              for (int ri = 0; ri < 2; ++ri)
                mma_sync16(acc[ri], ah[0], ah[1], ah[2], ah[3], bfh[ri][ks][0], bfh[ri][ks][1]);
            }
          }
          // P rows r0, r1 -> the MN-major z-stage operand (column cl, plane z, jt pair 2 t4)
#pragma unroll
          for (int ri = 0; ri < 2; ++ri)
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
              const int row = h2 ? r1 : r0;
              const int cl = j * p.cpt + row / Nz, z = row % Nz;
              uint32_t hv, lv;
              split2(rnd<TF>(acc[ri][2 * h2]), rnd<TF>(acc[ri][2 * h2 + 1]), hv, lv);
              const uint32_t off = (uint32_t)(cl * 2 + ri) * 128u + 4u * (uint32_t)t4 +
                                   (uint32_t)(z & 7) * 16u + (uint32_t)(z >> 3) * kg_a2;
              *reinterpret_cast<uint32_t*>(ah2 + off) = hv;
              if (SPLIT) *reinterpret_cast<uint32_t*>(ah2 + p.a2_bytes + off) = lv;
            }
        }
        mbar_arrive(&empty[s]);
        ++it;
      }
      if (!ok) break;
      fence_proxy_async();
      mbar_arrive(&a2full[gb]);
    }
    if (!ok) {
      atomicExch(p.err, 1);
      *sflag = 1;
    }
  } else {
    // ---------------- readback of D2 ----------------
    const int q = warp & 3;
    const int r = q * 32 + lane;  // TMEM lane = D2 row
    auto readback = [&](long long g, int gb) {
      // D2 row r -> T1 of column g*kG + r/16
      const long long col0 = g * kG;
      const int gcols = (int)min((long long)kG, p.ncol - col0);
      const int cl = r >> 4, ri = (r >> 3) & 1, jt = r & 7;
      const bool store = ri == 0 && cl < gcols && jt < Jt;
      float2* dst = p.out + ((col0 + cl) * Jz) * Jt + jt;
      for (int c0 = 0; c0 < p.N2; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)gb * (uint32_t)p.N2 + (uint32_t)c0, v);
        tmem_ld_wait();
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float own_r = __uint_as_float(v[2 * u]), own_i = __uint_as_float(v[2 * u + 1]);
          const float par_r = __shfl_xor_sync(0xffffffffu, own_r, 8);
          const float par_i = __shfl_xor_sync(0xffffffffu, own_i, 8);
          const int jz = (c0 >> 1) + u;
          if (store && jz < Jz) dst[(long long)jz * Jt] = make_float2(own_r - par_i, par_r + own_i);
        }
      }
    };
    long long gl = 0;
    bool ok = true;
    for (long long g = blockIdx.x; g < p.ngroups; g += gridDim.x, ++gl) {
      const int gb = (int)(gl & 1);
      if (!mbar_wait(&zdone[gb], (uint32_t)((gl >> 1) & 1), kWaitCycles) || *sflag) {
        ok = false;
        break;
      }
      fence_after_sync();
      readback(g, gb);
      fence_before_sync();
      mbar_arrive(&d2empty[gb]);
    }
    if (!ok) {
      atomicExch(p.err, 1);
      *sflag = 1;
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1) tmem_dealloc(tbase, p.tmem_cols);
}

static bool fwd_tz_plan(const Dims& d, bool split, FwdTcK& k, size_t& smem, char* why, size_t nwhy) {
  auto no = [&](const char* m) {
    if (why) snprintf(why, nwhy, "tensor-core t,z stage: %s", m);
    return false;
  };
  if (d.Nz != 16 && d.Nz != 32 && d.Nz != 64 && d.Nz != 128) return no("Nz must be 16, 32, 64 or 128");
  if (d.Nt % 8 != 0 || d.Nt > 64) return no("Nt must be a multiple of 8, at most 64");
  if (d.Jt > 8) return no("mt must be <= 8");
  if (2 * d.Jz > 128) return no("4*mz must be <= 128");
  k.Nz = (int)d.Nz;
  k.Nt = (int)d.Nt;
  k.Jz = (int)d.Jz;
  k.Jt = (int)d.Jt;
  k.cpt = (int)(128 / d.Nz);
  k.tpg = kG / k.cpt;
  k.KS = (int)(up((uint32_t)d.Nt, 16) / 16);
  k.N2 = (int)up((uint32_t)(2 * d.Jz), 16);
  k.tmem_cols = pow2_cols(2u * (uint32_t)k.N2);
  k.xf_bytes = (uint32_t)(128 * d.Nt * 4);
  k.a2_bytes = (uint32_t)(d.Nz / 8) * 2048u;
  k.a2_stride = (split ? 2u : 1u) * k.a2_bytes;
  k.b2_bytes = (uint32_t)(k.N2 * d.Nz * 2);
  for (int S = 10; S >= 2; --S) {
    uint32_t off = 0;
    k.o_xf = off;
    off += (uint32_t)S * k.xf_bytes;
    k.o_a2 = off = up(off, 1024);
    off += 2 * k.a2_stride;
    k.o_b2 = off = up(off, 128);
    off += 2 * k.b2_bytes;
    k.o_bar = off = up(off, 16);
    off += (uint32_t)(2 * S + 6) * 8 + 16;
    if (off <= 227 * 1024) {
      k.S = S;
      smem = off;
      return true;
    }
  }
  return no("shared memory does not fit");
}

bool fwd_tz_tc_supported(const Dims& d, char* why, size_t nwhy) {
  FwdTcK k{};
  size_t smem = 0;
  return fwd_tz_plan(d, true, k, smem, why, nwhy);
}

cudaError_t launch_fwd_tz_tc(const float* in, float2* out, int64_t ncol, const Dims& d,
                             const float2* ft, const float2* fz, bool split, bool tf32, int* err,
                             cudaStream_t s) {
  if (ncol <= 0) return cudaSuccess;
  FwdTcK k{};
  size_t smem = 0;
  if (!fwd_tz_plan(d, split || tf32, k, smem, nullptr, 0)) return cudaErrorInvalidValue;
  k.in = in;
  k.out = out;
  k.Ft = ft;
  k.Fz = fz;
  k.err = err;
  k.ncol = ncol;
  k.ngroups = (ncol + kG - 1) / kG;
  const void* kern = tf32 ? (const void*)k_fwd_tz_tc<true, true>
                          : (split ? (const void*)k_fwd_tz_tc<true, false> : (const void*)k_fwd_tz_tc<false, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<long long>(k.ngroups, sm_count());
  if (tf32)
    FNO_LAUNCH("fno_fwd_tz_tc_tf32", (k_fwd_tz_tc<true, true>), grid, kFwdThreads, smem, s, k);
  else if (split)
    FNO_LAUNCH("fno_fwd_tz_tc_bf16x3", (k_fwd_tz_tc<true, false>), grid, kFwdThreads, smem, s, k);
  else
    FNO_LAUNCH("fno_fwd_tz_tc_bf16", (k_fwd_tz_tc<false, false>), grid, kFwdThreads, smem, s, k);
  return cudaSuccess;
}

}  // namespace fno
