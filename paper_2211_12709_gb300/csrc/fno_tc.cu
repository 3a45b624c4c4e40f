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
// Warp roles (320 threads): warp 0 producer (bulk copies of 128-row tiles into a
// ring), warp 1 MMA issuer, warps 2-5 converters (fp32 tile -> BF16 hi/lo t-stage
// operand), warps 6-9 z-stage warps (D1 in TMEM -> MN-major z-stage operand in
// shared memory; D2 -> T1 in global memory).  Roles hand work to each other
// through mbarriers only.
//
// z-stage GEMM of a group of kG = 8 columns:
//   rows m = col * 16 + ri * 8 + jt   (P_re rows, then P_im rows, jt padded to 8)
//   cols n = 2 * jz + f                (f = 0: cos rows of Fz, f = 1: -sin rows)
//   D2[m][n] = sum_z P_ri[col][z][jt] * F_f[jz][z]
//   T_re = D2[(col,0,jt)][(jz,0)] - D2[(col,1,jt)][(jz,1)]
//   T_im = D2[(col,1,jt)][(jz,0)] + D2[(col,0,jt)][(jz,1)]
constexpr int kG = 8;
constexpr int kFwdThreads = 320;

struct FwdTcK {
  const float* in;
  float2* out;
  const float2* Ft;  // [Jt][Nt]  (cos, -sin) * scale
  const float2* Fz;  // [Jz][Nz]  (cos, -sin)
  int* err;
  long long ncol, ngroups;
  int Nz, Nt, Jz, Jt, cpt, tpg, K1, N2, S;
  uint32_t o_xf, xf_bytes, o_a1, a1_bytes, o_b1, b1_bytes, o_a2, a2_bytes, o_b2, b2_bytes, o_bar;
  uint32_t tmem_cols, d1_cols, d2_col;
};

template <bool SPLIT>
__global__ void __launch_bounds__(kFwdThreads, 1) k_fwd_tz_tc(const FwdTcK p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* xf = sm + p.o_xf;
  unsigned char* a1 = sm + p.o_a1;
  unsigned char* b1 = sm + p.o_b1;
  unsigned char* a2 = sm + p.o_a2;
  unsigned char* b2 = sm + p.o_b2;
  const int S = p.S;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + p.o_bar);
  uint64_t* empty = full + S;
  uint64_t* a1full = empty + S;
  uint64_t* a1empty = a1full + 2;
  uint64_t* d1full = a1empty + 2;
  uint64_t* d1empty = d1full + 2;
  uint64_t* a2full = d1empty + 2;
  uint64_t* zdone = a2full + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(zdone + 1);
  volatile int* sflag = reinterpret_cast<volatile int*>(tslot + 1);
  const int Nz = p.Nz, Nt = p.Nt, Jz = p.Jz, Jt = p.Jt;
  const uint32_t sbo1 = (uint32_t)p.K1 * 16u;   // K-major, K1/8 chunks of 128 B per row group
  const uint32_t sbo_b2 = (uint32_t)Nz * 16u;
  const uint32_t kg_a2 = 2048u;                  // MN-major: K group stride (16 row groups of 128 B)

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 128);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&a1full[b], 128);
      mbar_init(&a1empty[b], 1);
      mbar_init(&d1full[b], 1);
      mbar_init(&d1empty[b], 128);
    }
    mbar_init(a2full, 128);
    mbar_init(zdone, 1);
    *sflag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tslot, p.tmem_cols);
    tmem_relinquish();
  }
  for (uint32_t e = tid; e < p.a1_bytes * 4u / 16u; e += kFwdThreads)
    reinterpret_cast<uint4*>(a1)[e] = make_uint4(0, 0, 0, 0);
  for (uint32_t e = tid; e < p.a2_bytes * 2u / 16u; e += kFwdThreads)
    reinterpret_cast<uint4*>(a2)[e] = make_uint4(0, 0, 0, 0);
  for (int e = tid; e < 16 * p.K1; e += kFwdThreads) {
    const int n = e / p.K1, k = e - n * p.K1;
    const int ri = n >> 3, jt = n & 7;
    float v = 0.f;
    if (jt < Jt && k < Nt) {
      const float2 f = p.Ft[jt * Nt + k];
      v = ri ? f.y : f.x;
    }
    __nv_bfloat16 h, l;
    split1(v, h, l);
    const uint32_t off = koff(n, k, sbo1, 128);
    *reinterpret_cast<__nv_bfloat16*>(b1 + off) = h;
    *reinterpret_cast<__nv_bfloat16*>(b1 + p.b1_bytes + off) = l;
  }
  for (int e = tid; e < p.N2 * Nz; e += kFwdThreads) {
    const int n = e / Nz, z = e - n * Nz;
    float v = 0.f;
    if (n < 2 * Jz) {
      const float2 f = p.Fz[(n >> 1) * Nz + z];
      v = (n & 1) ? f.y : f.x;
    }
    __nv_bfloat16 h, l;
    split1(v, h, l);
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
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idt = idesc(kFmtBF16, 128, 16);
      const uint32_t idz = idesc(kFmtBF16, 128, p.N2) | (1u << 15);  // A2 is MN-major
      long long it = 0;
      long long gl = 0;
      bool ok = true;
      auto z_mma = [&](long long k) -> bool {
        if (!mbar_wait(a2full, (uint32_t)(k & 1), kWaitCycles)) return false;
        fence_after_sync();
        const uint32_t d = tbase + p.d2_col;
        const uint32_t sa = smem_u32(a2), sb = smem_u32(b2);
        for (int ks = 0; ks < Nz / 16; ++ks) {
          const uint64_t ah = sdesc(sa + (uint32_t)ks * 2u * kg_a2, kg_a2, 128);
          const uint64_t bh = sdesc(sb + (uint32_t)ks * 256u, 128, sbo_b2);
          mma_bf16(d, ah, bh, idz, ks > 0 ? 1u : 0u);
          if (SPLIT) {
            mma_bf16(d, ah, sdesc(sb + p.b2_bytes + (uint32_t)ks * 256u, 128, sbo_b2), idz, 1u);
            mma_bf16(d, sdesc(sa + p.a2_bytes + (uint32_t)ks * 2u * kg_a2, kg_a2, 128), bh, idz, 1u);
          }
        }
        mma_commit(zdone);
        return true;
      };
      for (long long g = blockIdx.x; g < p.ngroups && ok; g += gridDim.x, ++gl) {
        const int gb = (int)(gl & 1);
        const long long col0 = g * kG;
        const int gcols = (int)min((long long)kG, p.ncol - col0);
        const int ntile = (gcols + p.cpt - 1) / p.cpt;
        if (!mbar_wait(&d1empty[gb], (uint32_t)(((gl >> 1) & 1) ^ 1), kWaitCycles)) { ok = false; break; }
        for (int j = 0; j < ntile; ++j) {
          const int b = (int)(it & 1);
          if (!mbar_wait(&a1full[b], (uint32_t)((it >> 1) & 1), kWaitCycles)) { ok = false; break; }
          fence_after_sync();
          const uint32_t d = tbase + (uint32_t)gb * p.d1_cols + (uint32_t)j * 16u;
          const uint32_t sa = smem_u32(a1 + (size_t)b * 2 * p.a1_bytes), sb = smem_u32(b1);
          for (int ks = 0; ks < p.K1 / 16; ++ks) {
            const uint32_t ko = (uint32_t)ks * 256u;
            const uint64_t ah = sdesc(sa + ko, 128, sbo1), bh = sdesc(sb + ko, 128, sbo1);
            mma_bf16(d, ah, bh, idt, ks > 0 ? 1u : 0u);
            if (SPLIT) {
              mma_bf16(d, ah, sdesc(sb + p.b1_bytes + ko, 128, sbo1), idt, 1u);
              mma_bf16(d, sdesc(sa + p.a1_bytes + ko, 128, sbo1), bh, idt, 1u);
            }
          }
          mma_commit(&a1empty[b]);
          ++it;
        }
        if (!ok) break;
        mma_commit(&d1full[gb]);
        if (gl >= 1 && !z_mma(gl - 1)) { ok = false; break; }
        if (*sflag) { ok = false; break; }
      }
      if (ok && gl >= 1 && !z_mma(gl - 1)) ok = false;
      if (!ok) {
        atomicExch(p.err, 1);
        *sflag = 1;
      }
      // every issued MMA must be complete before TMEM is released
      if (gl >= 1) mbar_wait(zdone, (uint32_t)((gl - 1) & 1), kWaitCycles);
    }
  } else if (warp < 6) {
    // ---------------- converters ----------------
    const int ct = tid - 64;
    const int nch = Nt / 8;
    long long it = 0;
    bool ok = true;
    for (long long g = blockIdx.x; g < p.ngroups && ok; g += gridDim.x) {
      const long long col0 = g * kG;
      const int gcols = (int)min((long long)kG, p.ncol - col0);
      const int ntile = (gcols + p.cpt - 1) / p.cpt;
      for (int j = 0; j < ntile; ++j) {
        const int s = (int)(it % S), b = (int)(it & 1);
        const long long tc0 = col0 + (long long)j * p.cpt;
        const int rows = (int)min((long long)p.cpt, p.ncol - tc0) * Nz;
        if (!mbar_wait(&full[s], (uint32_t)((it / S) & 1), kWaitCycles) ||
            !mbar_wait(&a1empty[b], (uint32_t)(((it >> 1) & 1) ^ 1), kWaitCycles) || *sflag) {
          ok = false;
          break;
        }
        const float* xs = reinterpret_cast<const float*>(xf + (size_t)s * p.xf_bytes);
        unsigned char* ah = a1 + (size_t)b * 2 * p.a1_bytes;
        for (int e = ct; e < 128 * nch; e += 128) {
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
        fence_proxy_async();
        mbar_arrive(&empty[s]);
        mbar_arrive(&a1full[b]);
        ++it;
      }
    }
    if (!ok) {
      atomicExch(p.err, 1);
      *sflag = 1;
    }
  } else {
    // ---------------- z-stage warps ----------------
    const int q = warp & 3;
    const int r = q * 32 + lane;  // TMEM lane of this thread
    long long gl = 0;
    bool ok = true;
    auto readback = [&](long long g) {
      // D2 row r -> T1 of column g*kG + r/16
      const long long col0 = g * kG;
      const int gcols = (int)min((long long)kG, p.ncol - col0);
      const int cl = r >> 4, ri = (r >> 3) & 1, jt = r & 7;
      const bool store = ri == 0 && cl < gcols && jt < Jt;
      float2* dst = p.out + ((col0 + cl) * Jz) * Jt + jt;
      for (int c0 = 0; c0 < p.N2; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(tbase + ((uint32_t)(q * 32) << 16) + p.d2_col + (uint32_t)c0, v);
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
    for (long long g = blockIdx.x; g < p.ngroups; g += gridDim.x, ++gl) {
      const int gb = (int)(gl & 1);
      const long long col0 = g * kG;
      const int gcols = (int)min((long long)kG, p.ncol - col0);
      const int ntile = (gcols + p.cpt - 1) / p.cpt;
      if (!mbar_wait(&d1full[gb], (uint32_t)((gl >> 1) & 1), kWaitCycles) || *sflag) { ok = false; break; }
      if (gl >= 1) {
        if (!mbar_wait(zdone, (uint32_t)((gl - 1) & 1), kWaitCycles)) { ok = false; break; }
        fence_after_sync();
        readback(g - gridDim.x);
      }
      fence_after_sync();
      for (int j = 0; j < ntile; ++j) {
        uint32_t v[16];
        tmem_ld16(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)gb * p.d1_cols + (uint32_t)j * 16u, v);
        tmem_ld_wait();
        const int cl = j * p.cpt + r / Nz;
        const int z = r % Nz;
        if (cl < gcols) {
#pragma unroll
          for (int ri = 0; ri < 2; ++ri) {
            float x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = __uint_as_float(v[ri * 8 + u]);
            uint4 h, l;
            if (SPLIT) {
              split2(x[0], x[1], h.x, l.x);
              split2(x[2], x[3], h.y, l.y);
              split2(x[4], x[5], h.z, l.z);
              split2(x[6], x[7], h.w, l.w);
            } else {
              h = make_uint4(bf2(x[0], x[1]), bf2(x[2], x[3]), bf2(x[4], x[5]), bf2(x[6], x[7]));
            }
            const uint32_t off = (uint32_t)(cl * 2 + ri) * 128u + (uint32_t)(z & 7) * 16u + (uint32_t)(z >> 3) * kg_a2;
            *reinterpret_cast<uint4*>(a2 + off) = h;
            if (SPLIT) *reinterpret_cast<uint4*>(a2 + p.a2_bytes + off) = l;
          }
        }
      }
      fence_before_sync();
      fence_proxy_async();
      mbar_arrive(a2full);
      mbar_arrive(&d1empty[gb]);
    }
    if (ok && gl >= 1) {
      if (mbar_wait(zdone, (uint32_t)((gl - 1) & 1), kWaitCycles)) {
        fence_after_sync();
        readback(blockIdx.x + (gl - 1) * gridDim.x);
      } else {
        ok = false;
      }
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

static bool fwd_tz_plan(const Dims& d, FwdTcK& k, size_t& smem, char* why, size_t nwhy) {
  auto no = [&](const char* m) {
    if (why) snprintf(why, nwhy, "tensor-core t,z stage: %s", m);
    return false;
  };
  if (d.Nz != 16 && d.Nz != 32 && d.Nz != 64 && d.Nz != 128) return no("Nz must be 16, 32, 64 or 128");
  if (d.Nt % 8 != 0 || d.Nt > 64) return no("Nt must be a multiple of 8, at most 64");
  if (d.Jt > 8) return no("mt must be <= 8");
  if (2 * d.Jz > 128) return no("2*mz must be <= 64");
  k.Nz = (int)d.Nz;
  k.Nt = (int)d.Nt;
  k.Jz = (int)d.Jz;
  k.Jt = (int)d.Jt;
  k.cpt = (int)(128 / d.Nz);
  k.tpg = kG / k.cpt;
  k.K1 = (int)up((uint32_t)d.Nt, 16);
  k.N2 = (int)up((uint32_t)(2 * d.Jz), 16);
  k.d1_cols = (uint32_t)(k.tpg * 16);
  k.d2_col = 2 * k.d1_cols;
  k.tmem_cols = pow2_cols(k.d2_col + (uint32_t)k.N2);
  if (k.tmem_cols > 512) return no("too many TMEM columns");
  k.xf_bytes = (uint32_t)(128 * d.Nt * 4);
  k.a1_bytes = (uint32_t)(128 * k.K1 * 2);
  k.b1_bytes = (uint32_t)(16 * k.K1 * 2);
  k.a2_bytes = (uint32_t)(d.Nz / 8) * 2048u;
  k.b2_bytes = (uint32_t)(k.N2 * d.Nz * 2);
  for (int S = 6; S >= 2; --S) {
    uint32_t off = 0;
    k.o_xf = off;
    off += (uint32_t)S * k.xf_bytes;
    k.o_a1 = off = up(off, 1024);
    off += 4 * k.a1_bytes;
    k.o_b1 = off = up(off, 128);
    off += 2 * k.b1_bytes;
    k.o_a2 = off = up(off, 1024);
    off += 2 * k.a2_bytes;
    k.o_b2 = off = up(off, 128);
    off += 2 * k.b2_bytes;
    k.o_bar = off = up(off, 16);
    off += (uint32_t)(2 * S + 10) * 8 + 16;
    if (off <= 227 * 1024) {
      k.S = S;
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
  k.ngroups = (ncol + kG - 1) / kG;
  const void* kern = split ? (const void*)k_fwd_tz_tc<true> : (const void*)k_fwd_tz_tc<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<long long>(k.ngroups, sm_count());
  if (split)
    FNO_LAUNCH_TC("fno_fwd_tz_tc_bf16x3", k_fwd_tz_tc<true>, grid, kFwdThreads, smem, s, k);
  else
    FNO_LAUNCH_TC("fno_fwd_tz_tc_bf16", k_fwd_tz_tc<false>, grid, kFwdThreads, smem, s, k);
  return cudaSuccess;
}

// ============================================================================
// Inverse z, t stages + epilogue
// ============================================================================
// Warp roles (448 threads): warp 0 producer (bulk copies of the linear input
// of each 128-point tile), warp 1 MMA issuer, warps 2-5 operand builders
// (A_X from the staged input, B_S = inverse z stage of the column spectrum,
// and -- for the dA pass -- A_w = x^T), warps 6-13 epilogue (TMEM -> outputs;
// for the dA pass also dA as the MN-major operand of dW_lin).  Double-buffered
// operands and accumulators; mbarrier hand-offs only.
//
// Inverse z stage with +-k pairing (kept kz = -mz..mz-1):
//   Q(z) = sum_{k=0..mz} E_k cos(k th) + i sum_{k=1..mz} O_k sin(k th),  th = 2 pi z / Nz
//   E_0 = U_0, E_k = U_k + U_-k, O_k = U_k - U_-k (0 < k < mz), E_mz = U_-mz, O_mz = -U_-mz
constexpr int kEpiThreads = 448;
constexpr int kMzMax = 16;

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
  int Nz, Nt, Jz, Jt, mz, Cs, Cl, w_si, w_sc;
  int zc, P, PS, nzc, NP, KX, KS, S, GW;  // GW: row groups of A_w holding real rows (DA)
  uint32_t o_aw, aw_bytes, o_xf, xf_bytes, o_ax, ax_bytes, o_bx, bx_bytes, o_as, as_bytes;
  uint32_t o_bs, bs_bytes, o_bw, bw_bytes, o_eo, o_cs, o_bias, o_bar;
  uint32_t tmem_cols;
};

template <int MODE, bool SPLIT>
__global__ void __launch_bounds__(kEpiThreads, 1) k_epi_tc(const EpiTcK p) {
  constexpr bool LIN = MODE != EPI_SPECTRAL;
  constexpr bool DA = MODE == EPI_DA;
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* aw = sm + p.o_aw;   // [2][hi, lo]   (DA)
  float* xf = reinterpret_cast<float*>(sm + p.o_xf);
  unsigned char* ax = sm + p.o_ax;   // [2][hi, lo]
  unsigned char* bx = sm + p.o_bx;   // [hi, lo]
  unsigned char* as_ = sm + p.o_as;  // [hi, lo]
  unsigned char* bs = sm + p.o_bs;   // [2][hi, lo]
  unsigned char* bw = sm + p.o_bw;   // [2][hi, lo]   (DA)
  float4* eo = reinterpret_cast<float4*>(sm + p.o_eo);  // [Cs][Jt][mz+1] (E, O)
  float2* cs = reinterpret_cast<float2*>(sm + p.o_cs);  // [Nz][mz+1] (cos, sin)
  float* sbias = reinterpret_cast<float*>(sm + p.o_bias);
  const int S = p.S;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + p.o_bar);
  uint64_t* empty = full + S;
  uint64_t* opfull = empty + S;
  uint64_t* opempty = opfull + 2;
  uint64_t* accfull = opempty + 2;
  uint64_t* accempty = accfull + 2;
  uint64_t* bwfull = accempty + 2;
  uint64_t* bwempty = bwfull + 2;
  uint64_t* wdone = bwempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(wdone + 1);
  volatile int* sflag = reinterpret_cast<volatile int*>(tslot + 1);
  const int Nz = p.Nz, Nt = p.Nt, Jz = p.Jz, Jt = p.Jt, mz = p.mz, Cs = p.Cs, Cl = p.Cl;
  const int P = p.P, PS = p.PS, NP = p.NP, KX = p.KX, KS = p.KS;
  const uint32_t sbo_x = (uint32_t)KX * 16u, sbo_s = (uint32_t)KS * 16u;
  const uint32_t band_bytes = (uint32_t)NP * (uint32_t)KS * 2u;
  const uint32_t sbo_w = (uint32_t)P * 16u;          // A_w: K = P points
  const uint32_t kg_w = (uint32_t)(NP / 8) * 128u;   // B_w (MN-major): K group stride
  const long long chan = p.NxNy * (long long)Nz * Nt;
  const long long t_begin = p.ntiles * blockIdx.x / gridDim.x;
  const long long t_end = p.ntiles * (blockIdx.x + 1) / gridDim.x;
  const int nloc = (int)(t_end - t_begin);

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 128);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&opfull[b], 128);
      mbar_init(&opempty[b], 1);
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], 256);
      mbar_init(&bwfull[b], 256);
      mbar_init(&bwempty[b], 1);
    }
    mbar_init(wdone, 1);
    *sflag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tslot, p.tmem_cols);
    tmem_relinquish();
  }
  // constant operands, zero padding
  for (uint32_t e = tid; e < 4u * p.ax_bytes / 16u; e += kEpiThreads) reinterpret_cast<uint4*>(ax)[e] = make_uint4(0, 0, 0, 0);
  for (uint32_t e = tid; e < 4u * p.bs_bytes / 16u; e += kEpiThreads) reinterpret_cast<uint4*>(bs)[e] = make_uint4(0, 0, 0, 0);
  if (DA) {
    for (uint32_t e = tid; e < 4u * p.aw_bytes / 16u; e += kEpiThreads) reinterpret_cast<uint4*>(aw)[e] = make_uint4(0, 0, 0, 0);
    for (uint32_t e = tid; e < 4u * p.bw_bytes / 16u; e += kEpiThreads) reinterpret_cast<uint4*>(bw)[e] = make_uint4(0, 0, 0, 0);
  }
  if (LIN) {
    for (int e = tid; e < NP * KX; e += kEpiThreads) {
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
    for (int e = tid; e < rows * KS; e += kEpiThreads) {
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
  for (int e = tid; e < Nz * (mz + 1); e += kEpiThreads) {
    const int z = e / (mz + 1), k = e - z * (mz + 1);
    const float2 f = p.Iz[z * Jz + k];  // jz = k: kz = k for k < mz, kz = -mz for k = mz
    cs[e] = (k < mz) ? f : make_float2(f.x, -f.y);
  }
  if (MODE == EPI_FWD || MODE == EPI_DA)
    for (int c = tid; c < Cs; c += kEpiThreads) sbias[c] = p.bias[c];
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t dw_col = 2u * (uint32_t)NP;

  auto tile_geom = [&](int n, long long& b, long long& xy, int& z0, int& zn) {
    const long long tau = t_begin + n;
    const long long col = tau / p.nzc;
    z0 = (int)(tau - col * p.nzc) * p.zc;
    zn = min(p.zc, Nz - z0);
    b = col / p.NxNy;
    xy = col - b * p.NxNy;
  };

  if (warp == 0) {
    // ---------------- producer ----------------
    if (LIN && lane == 0) {
      int it = 0;
      for (; it < nloc; ++it) {
        const int s = it % S;
        if (!mbar_wait(&empty[s], (uint32_t)(((it / S) & 1) ^ 1), kWaitCycles) || *sflag) {
          atomicExch(p.err, 1);
          *sflag = 1;
          break;
        }
        long long b, xy;
        int z0, zn;
        tile_geom(it, b, xy, z0, zn);
        const uint32_t bytes = (uint32_t)(zn * Nt * 4);
        mbar_arrive_expect_tx(&full[s], bytes * (uint32_t)Cl);
        for (int i = 0; i < Cl; ++i) {
          const float* src = p.lin + (b * Cl + i) * chan + xy * (long long)(Nz * Nt) + (long long)z0 * Nt;
          bulk_g2s(xf + ((size_t)s * Cl + i) * PS, src, bytes, &full[s]);
        }
      }
      for (int k = (it > S ? it - S : 0); k < it; ++k)
        mbar_wait(&full[k % S], (uint32_t)((k / S) & 1), kWaitCycles);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idv = idesc(kFmtBF16, 128, NP);
      const uint32_t idw = idesc(kFmtBF16, 128, NP) | (1u << 16);  // B_w is MN-major
      bool ok = true;
      auto dw_mma = [&](int k) -> bool {
        const int b = k & 1;
        if (!mbar_wait(&bwfull[b], (uint32_t)((k >> 1) & 1), kWaitCycles)) return false;
        fence_after_sync();
        const uint32_t sa = smem_u32(aw + (size_t)b * 2 * p.aw_bytes), sb = smem_u32(bw + (size_t)b * 2 * p.bw_bytes);
        const uint32_t dwd = tbase + dw_col + (uint32_t)(b * NP);
        for (int ks = 0; ks < P / 16; ++ks) {
          const uint64_t ah = sdesc(sa + (uint32_t)ks * 256u, 128, sbo_w);
          const uint64_t bh = sdesc(sb + (uint32_t)ks * 2u * kg_w, kg_w, 128);
          mma_bf16(dwd, ah, bh, idw, ks > 0 ? 1u : 0u);
          if (SPLIT) {
            mma_bf16(dwd, ah, sdesc(sb + p.bw_bytes + (uint32_t)ks * 2u * kg_w, kg_w, 128), idw, 1u);
            mma_bf16(dwd, sdesc(sa + p.aw_bytes + (uint32_t)ks * 256u, 128, sbo_w), bh, idw, 1u);
          }
        }
        mma_commit(&opempty[b]);
        mma_commit(&bwempty[b]);
        return true;
      };
      int n = 0;
      for (; n < nloc; ++n) {
        const int b = n & 1;
        long long bb, xy;
        int z0, zn;
        tile_geom(n, bb, xy, z0, zn);
        if (!mbar_wait(&opfull[b], (uint32_t)((n >> 1) & 1), kWaitCycles) ||
            !mbar_wait(&accempty[b], (uint32_t)(((n >> 1) & 1) ^ 1), kWaitCycles) || *sflag) {
          ok = false;
          break;
        }
        fence_after_sync();
        const uint32_t d = tbase + (uint32_t)(b * NP);
        uint32_t accf = 0;
        if (LIN) {
          const uint32_t sa = smem_u32(ax + (size_t)b * 2 * p.ax_bytes), sb = smem_u32(bx);
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
        const uint32_t sa = smem_u32(as_), sb = smem_u32(bs + (size_t)b * 2 * p.bs_bytes);
        for (int zz = 0; zz < zn; ++zz) {
          const uint32_t ao = ((uint32_t)(128 - Nt - zz * Nt) >> 3) * sbo_s;
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
        mma_commit(&accfull[b]);
        if (!DA) mma_commit(&opempty[b]);
        if (DA && n >= 1 && !dw_mma(n - 1)) {
          ok = false;
          break;
        }
      }
      if (DA && ok && n >= 1 && !dw_mma(n - 1)) ok = false;
      if (DA) mma_commit(wdone);
      if (!ok) {
        atomicExch(p.err, 1);
        *sflag = 1;
      }
      // all issued MMAs complete before TMEM is released
      if (DA) {
        mbar_wait(wdone, 0, kWaitCycles);
      } else if (n >= 1) {
        mbar_wait(&accfull[(n - 1) & 1], (uint32_t)(((n - 1) >> 1) & 1), kWaitCycles);
      }
    }
  } else if (warp < 6) {
    // ---------------- operand builders ----------------
    const int ot = tid - 64;
    long long cur_col = -1;
    bool ok = true;
    for (int n = 0; n < nloc; ++n) {
      const int b = n & 1, s = n % S;
      long long bb, xy;
      int z0, zn;
      tile_geom(n, bb, xy, z0, zn);
      const long long col = bb * p.NxNy + xy;
      if (col != cur_col) {
        named_sync(1, 128);  // previous tile's reads of eo are done
        const int JZT = Jz * Jt;
        for (int e = ot; e < Cs * Jt * (mz + 1); e += 128) {
          const int k = e % (mz + 1), jt = (e / (mz + 1)) % Jt, c = e / ((mz + 1) * Jt);
          const float2* u = p.U + ((bb * Cs + c) * p.NxNy + xy) * JZT + jt;
          float4 v;
          if (k == 0) {
            const float2 a = u[0];
            v = make_float4(a.x, a.y, 0.f, 0.f);
          } else if (k < mz) {
            const float2 a = u[k * Jt], m = u[(2 * mz - k) * Jt];
            v = make_float4(a.x + m.x, a.y + m.y, a.x - m.x, a.y - m.y);
          } else {
            const float2 m = u[mz * Jt];
            v = make_float4(m.x, m.y, -m.x, -m.y);
          }
          eo[e] = v;
        }
        named_sync(1, 128);
        cur_col = col;
      }
      if (!mbar_wait(&opempty[b], (uint32_t)(((n >> 1) & 1) ^ 1), kWaitCycles) ||
          (LIN && !mbar_wait(&full[s], (uint32_t)((n / S) & 1), kWaitCycles)) || *sflag) {
        ok = false;
        break;
      }
      const int valid = zn * Nt;
      if (LIN) {
        const float* xs = xf + (size_t)s * Cl * PS;
        unsigned char* axb = ax + (size_t)b * 2 * p.ax_bytes;
        const int ich = (Cl + 7) / 8;
        for (int e = ot; e < P * ich; e += 128) {
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
          *reinterpret_cast<uint4*>(axb + off) = h;
          if (SPLIT) *reinterpret_cast<uint4*>(axb + p.ax_bytes + off) = l;
        }
        if (DA) {
          // A_w = x^T (rows i, K = points) plus the ones row i = Cl (db)
          unsigned char* awb = aw + (size_t)b * 2 * p.aw_bytes;
          const int kch = P / 8;
          for (int e = ot; e < (Cl + 1) * kch; e += 128) {
            const int i = e / kch, c8 = e - i * kch;
            float v[8];
            if (i < Cl) {
              const float4 a0 = reinterpret_cast<const float4*>(xs + i * PS + c8 * 8)[0];
              const float4 a1 = reinterpret_cast<const float4*>(xs + i * PS + c8 * 8)[1];
              v[0] = a0.x; v[1] = a0.y; v[2] = a0.z; v[3] = a0.w;
              v[4] = a1.x; v[5] = a1.y; v[6] = a1.z; v[7] = a1.w;
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j) v[j] = 1.f;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (c8 * 8 + j >= valid) v[j] = 0.f;
            uint4 h, l;
            if (SPLIT) {
              split2(v[0], v[1], h.x, l.x);
              split2(v[2], v[3], h.y, l.y);
              split2(v[4], v[5], h.z, l.z);
              split2(v[6], v[7], h.w, l.w);
            } else {
              h = make_uint4(bf2(v[0], v[1]), bf2(v[2], v[3]), bf2(v[4], v[5]), bf2(v[6], v[7]));
            }
            const uint32_t off = koff(i, c8 * 8, sbo_w, 128);
            *reinterpret_cast<uint4*>(awb + off) = h;
            if (SPLIT) *reinterpret_cast<uint4*>(awb + p.aw_bytes + off) = l;
          }
        }
        mbar_arrive(&empty[s]);
      }
      // B_S: one band per z plane, row c, K = (jt, ri)
      {
        unsigned char* bsb = bs + (size_t)b * 2 * p.bs_bytes;
        for (int e = ot; e < Cs * Jt; e += 128) {
          const int jt = e % Jt, c = e / Jt;
          float4 r[kMzMax + 1];
          const float4* src = eo + (size_t)(c * Jt + jt) * (mz + 1);
#pragma unroll
          for (int k = 0; k <= kMzMax; ++k)
            if (k <= mz) r[k] = src[k];
          for (int zz = 0; zz < zn; ++zz) {
            const float2* cz = cs + (size_t)(z0 + zz) * (mz + 1);
            float qr = 0.f, qi = 0.f;
#pragma unroll
            for (int k = 0; k <= kMzMax; ++k) {
              if (k <= mz) {
                const float2 t = cz[k];
                qr = fmaf(r[k].x, t.x, qr);
                qr = fmaf(-r[k].w, t.y, qr);
                qi = fmaf(r[k].y, t.x, qi);
                qi = fmaf(r[k].z, t.y, qi);
              }
            }
            const uint32_t off = (uint32_t)zz * band_bytes + koff(c, 2 * jt, sbo_s, 128);
            if (SPLIT) {
              uint32_t h, l;
              split2(qr, qi, h, l);
              *reinterpret_cast<uint32_t*>(bsb + off) = h;
              *reinterpret_cast<uint32_t*>(bsb + p.bs_bytes + off) = l;
            } else {
              *reinterpret_cast<uint32_t*>(bsb + off) = bf2(qr, qi);
            }
          }
        }
      }
      fence_proxy_async();
      mbar_arrive(&opfull[b]);
    }
    if (!ok) {
      atomicExch(p.err, 1);
      *sflag = 1;
    }
  } else {
    // ---------------- epilogue warps ----------------
    const int q = warp & 3, half = (warp - 6) >> 2;
    const int row = q * 32 + lane;
    const int c_lo = half * (NP / 2);
    bool ok = true;
    // Kahan-compensated running sums of this thread's dW_lin / db row (q == 0 warps)
    float wsum[32], wcmp[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      wsum[j] = 0.f;
      wcmp[j] = 0.f;
    }
    auto fold = [&](int k) {
      // per-tile accumulator of tile k (complete) -> running sums
      if (!DA || q != 0) return;
#pragma unroll
      for (int c0 = 0; c0 < 32; c0 += 8) {
        if (c0 >= NP / 2) break;
        uint32_t v[8];
        tmem_ld8(tbase + dw_col + (uint32_t)((k & 1) * NP + c_lo + c0), v);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int idx = c0 + j;
          if (idx < 32) {
            const float y = __uint_as_float(v[j]) - wcmp[idx];
            const float t = wsum[idx] + y;
            wcmp[idx] = (t - wsum[idx]) - y;
            wsum[idx] = t;
          }
        }
      }
    };
    for (int n = 0; n < nloc; ++n) {
      const int b = n & 1;
      long long bb, xy;
      int z0, zn;
      tile_geom(n, bb, xy, z0, zn);
      if (!mbar_wait(&accfull[b], (uint32_t)((n >> 1) & 1), kWaitCycles) ||
          (DA && !mbar_wait(&bwempty[b], (uint32_t)(((n >> 1) & 1) ^ 1), kWaitCycles)) || *sflag) {
        ok = false;
        break;
      }
      fence_after_sync();
      if (DA && n >= 2) fold(n - 2);  // bwempty[b] certified that dW(n-2) is complete
      const int valid = zn * Nt;
      const bool rv = row < valid;
      const long long pofs = xy * (long long)(Nz * Nt) + (long long)z0 * Nt + row;
      const uint32_t ta = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * NP + c_lo);
      unsigned char* bwb = bw + (size_t)b * 2 * p.bw_bytes;
      for (int c0 = 0; c0 < NP / 2; c0 += 8) {
        uint32_t v[8];
        tmem_ld8(ta + (uint32_t)c0, v);
        tmem_ld_wait();
        float dav[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int o = c_lo + c0 + j;
          const float a = __uint_as_float(v[j]);
          dav[j] = 0.f;
          if (o < Cs && rv) {
            const long long oofs = (bb * Cs + o) * chan + pofs;
            if (MODE == EPI_FWD) {
              p.out[oofs] = gelu_f(a + sbias[o]);
            } else if (MODE == EPI_DA) {
              const float da = p.dz[oofs] * gelu_grad_f(a + sbias[o]);
              p.out[oofs] = da;
              dav[j] = da;
            } else {
              p.out[oofs] = a;
            }
          }
        }
        if (DA) {
          uint4 h, l;
          if (SPLIT) {
            split2(dav[0], dav[1], h.x, l.x);
            split2(dav[2], dav[3], h.y, l.y);
            split2(dav[4], dav[5], h.z, l.z);
            split2(dav[6], dav[7], h.w, l.w);
          } else {
            h = make_uint4(bf2(dav[0], dav[1]), bf2(dav[2], dav[3]), bf2(dav[4], dav[5]), bf2(dav[6], dav[7]));
          }
          const uint32_t off = (uint32_t)((c_lo + c0) >> 3) * 128u + (uint32_t)(row & 7) * 16u + (uint32_t)(row >> 3) * kg_w;
          *reinterpret_cast<uint4*>(bwb + off) = h;
          if (SPLIT) *reinterpret_cast<uint4*>(bwb + p.bw_bytes + off) = l;
        }
      }
      fence_before_sync();
      mbar_arrive(&accempty[b]);
      if (DA) {
        fence_proxy_async();
        mbar_arrive(&bwfull[b]);
      }
    }
    if (!ok) {
      atomicExch(p.err, 1);
      *sflag = 1;
    }
    if (DA) {
      // the last two per-tile accumulators, then per-CTA sums of dW_lin (rows i < Cl) and db (row Cl)
      const bool got = ok && mbar_wait(wdone, 0, kWaitCycles);
      fence_after_sync();
      if (got) {
        if (nloc >= 2) fold(nloc - 2);
        if (nloc >= 1) fold(nloc - 1);
      }
      const int npair = Cl * Cs + Cs;
      if (q == 0) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int o = c_lo + j;
          if (j < NP / 2 && o < Cs && row <= Cl) {
            const int idx = (row < Cl) ? row * Cs + o : Cl * Cs + o;
            p.part[(long long)blockIdx.x * npair + idx] = got ? wsum[j] - wcmp[j] : 0.f;
          }
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1) tmem_dealloc(tbase, p.tmem_cols);
}

int epilogue_tc_max_grid() { return 1024; }

static bool epi_plan(const Dims& d, int mode, int Cs, int Cl, EpiTcK& k, size_t& smem,
                     char* why, size_t nwhy) {
  auto no = [&](const char* m) {
    if (why) snprintf(why, nwhy, "tensor-core epilogue: %s", m);
    return false;
  };
  if (d.Nt % 8 != 0 || d.Nt > 128 || 128 % d.Nt != 0) return no("Nt must divide 128 and be a multiple of 8");
  if (2 * d.Jt > 32) return no("mt must be <= 16");
  if (d.mz > kMzMax) return no("mz must be <= 16");
  if (Cs > 64 || (mode != EPI_SPECTRAL && Cl > 64)) return no("channels must be <= 64");
  if (mode == EPI_DA && Cl + 1 > 32) return no("C_in must be <= 31 for the dW_lin tensor-core pass");
  k.Nz = (int)d.Nz;
  k.Nt = (int)d.Nt;
  k.Jz = (int)d.Jz;
  k.Jt = (int)d.Jt;
  k.mz = (int)d.mz;
  k.Cs = Cs;
  k.Cl = mode == EPI_SPECTRAL ? 0 : Cl;
  k.zc = (int)std::min<int64_t>(d.Nz, 128 / d.Nt);
  k.P = k.zc * (int)d.Nt;
  k.PS = k.P + 4;
  k.nzc = (int)((d.Nz + k.zc - 1) / k.zc);
  k.NP = (int)up((uint32_t)Cs, 16);
  k.KX = k.Cl > 0 ? (int)up((uint32_t)k.Cl, 16) : 0;
  k.KS = (int)up((uint32_t)(2 * d.Jt), 16);
  k.GW = (k.Cl + 1 + 7) / 8;
  k.tmem_cols = pow2_cols(2u * (uint32_t)k.NP + (mode == EPI_DA ? 2u * (uint32_t)k.NP : 0u));
  k.ax_bytes = (uint32_t)(128 * std::max(k.KX, 16) * 2);
  k.bx_bytes = (uint32_t)(k.NP * std::max(k.KX, 16) * 2);
  k.as_bytes = (uint32_t)((256 - d.Nt) * k.KS * 2);
  k.bs_bytes = (uint32_t)(k.zc * k.NP * k.KS * 2);
  // A_w: GW real row groups; the MMA also reads (junk) groups up to 16, which must
  // stay inside the allocation, so A_w sits at the start of shared memory.
  k.aw_bytes = mode == EPI_DA ? (uint32_t)k.GW * (uint32_t)k.P * 16u : 0u;
  k.bw_bytes = mode == EPI_DA ? (uint32_t)(k.P / 8) * (uint32_t)(k.NP / 8) * 128u : 0u;
  k.xf_bytes = (uint32_t)(std::max(k.Cl, 1) * k.PS * 4);
  for (int S = 4; S >= 2; --S) {
    uint32_t off = 0;
    k.o_aw = off;
    off += 4 * k.aw_bytes;
    k.o_xf = off = up(off, 128);
    off += (uint32_t)S * k.xf_bytes;
    k.o_ax = off = up(off, 128);
    off += 4 * k.ax_bytes;
    k.o_bx = off = up(off, 128);
    off += 2 * k.bx_bytes;
    k.o_as = off = up(off, 128);
    off += 2 * k.as_bytes;
    k.o_bs = off = up(off, 128);
    off += 4 * k.bs_bytes;
    k.o_bw = off = up(off, 128);
    off += 4 * k.bw_bytes;
    k.o_eo = off = up(off, 16);
    off += (uint32_t)(Cs * d.Jt * (d.mz + 1) * 16);
    k.o_cs = off = up(off, 16);
    off += (uint32_t)(d.Nz * (d.mz + 1) * 8);
    k.o_bias = off = up(off, 16);
    off += (uint32_t)(Cs * 4);
    k.o_bar = off = up(off, 16);
    off += (uint32_t)(2 * S + 13) * 8 + 16;
    // the junk rows of the A_w MMA read up to 16 row groups past o_aw
    const uint32_t junk_end = mode == EPI_DA ? 16u * (uint32_t)k.P * 16u + 3u * k.aw_bytes : 0u;
    if (off <= 227 * 1024 && junk_end <= off) {
      k.S = S;
      smem = off;
      return true;
    }
  }
  return no("shared memory does not fit");
}

bool epilogue_tc_supported(const Dims& d, int mode, int Cs, int Cl, char* why, size_t nwhy) {
  EpiTcK k{};
  size_t smem = 0;
  return epi_plan(d, mode, Cs, Cl, k, smem, why, nwhy);
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
  FNO_LAUNCH_TC(names[SPLIT ? 1 : 0][MODE], (k_epi_tc<MODE, SPLIT>), grid, kEpiThreads, smem, s, k);
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
  if (!epi_plan(d, a.mode, a.Cs, a.Cl, k, smem, nullptr, 0)) return cudaErrorInvalidValue;
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
  int grid = (int)std::min<long long>(k.ntiles, (long long)sm_count());
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
