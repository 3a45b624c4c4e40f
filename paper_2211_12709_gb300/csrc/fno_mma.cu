// fno_mma.cu -- inverse z, t stages fused with the pointwise epilogue on the
// tensor cores through warp-level mma.sync (BF16 or split BF16, FP32
// accumulation): the last stage of the inverse transform of Alg. 2 (Sec. IV-C)
// with the 1x1 bypass, bias and GELU of the block, and in its dA mode the
// dW_lin / db reductions of the backward pass.
//
// Where this kernel runs: plain BF16 (one product per stage, so the tcgen05
// form's operand conversion costs more than it saves), the dA mode of the
// recomputing backward, and shapes outside the tcgen05 epilogue's tiling.
// mma.sync m16n8k16 sustains about 1020 BF16 MAC/clk/SM on this GPU (FP32
// FFMA: 117), keeps operands and accumulators in registers, and feeds the GELU
// epilogue without a TMEM round trip; a tcgen05.mma of M = 128 at the N <= 32
// of these contractions runs at most 1.6 times that rate.
//
// A tile is 128 points of one (b, x, y) column: ZB = 128 / Nt z-planes.  Each
// of the 8 warps owns one m-tile of 16 consecutive points.  Per tile:
//   stage 1 (inverse z, complex, as a real GEMM)
//     Q[(o, jt)][(z, re/im)] = sum_k U'[(o, jt)][k] Bz[k][(z, re/im)],
//     k = (jz, re/im); A = U' (the column's spectrum in shared memory, rebuilt
//     when the column changes), B = basis fragments from a global table.
//   stage 2 (inverse t) + stage 3 (1x1):
//     acc[p = (z, t)][o] = bias[o] + sum_k2 Tb[t][k2] Q[z][o][k2]
//                                  + sum_i  X[i][p] Wl[i][o]
//     k2 = (re/im, jt); Tb holds c(kt)/N cos and -c(kt)/N sin.
//   epilogue: FWD z = GELU(acc); DA dA = dz GELU'(acc); DX, SPECTRAL out = acc.
//   stage 5 (DA only): dWl[i][o] (+ db through a row of ones) += X[i][:] . dA[o][:]
//     over the tile's points, Kahan-folded per tile.
// The x tile arrives by bulk copy (TMA engine), one tile ahead.
// Precision.  BF16: one product everywhere.  Split BF16: the DFT stages (1, 2)
// use a = hi + lo with products hi.hi + hi.lo + lo.hi; the 1x1 contractions
// (3, 5), which carry the bypass term that dominates the block output, split
// both operands in three BF16 parts (exact for FP32 inputs) and sum the six
// products of order >= 2^-16, so they are as accurate as FP32 products.
// GELU uses the erf approximation 7.1.26 of Abramowitz and Stegun (absolute
// error below 1.5e-7) with hardware exp2 and reciprocal.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include <cstdio>

#include "fno_internal.h"
#include "warp_mma.h"
#include "tma.h"

namespace fno {

namespace {

constexpr int kP = 128;        // points per tile
constexpr int kWarps = 8;      // one 16-point m-tile per warp
constexpr int kThreads = 32 * kWarps;
constexpr int kNTM = 4;        // max n-tiles of 8 output channels (Cs <= 32)
constexpr int kClMax = 32;     // max 1x1 input channels
constexpr int kKZMax = 3;      // stage-1 k-steps (2 * mz <= 24)

// ---- warp-level tensor-core helpers (inline PTX) ----------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void ldsm_x4(uint32_t a, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                        uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t a, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                          uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t a, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
               : "=r"(r0), "=r"(r1)
               : "r"(a));
}
__device__ __forceinline__ void stsm_x4_t(uint32_t a, uint32_t r0, uint32_t r1, uint32_t r2,
                                          uint32_t r3) {
  asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1,%2,%3,%4};" ::"r"(a),
               "r"(r0), "r"(r1), "r"(r2), "r"(r3)
               : "memory");
}
// D += A (16x16, row) * B (16x8, col), BF16 in, FP32 accumulate
__device__ __forceinline__ void mma16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                      uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// D += A (16x8, row) * B (8x8, col)
__device__ __forceinline__ void mma8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0));
}

// hi/lo BF16 split of two floats, packed in pairs (first value in the low half)
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void ldsm_x2(uint32_t a, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
               : "=r"(r0), "=r"(r1)
               : "r"(a));
}
__device__ __forceinline__ void stsm_x2_t(uint32_t a, uint32_t r0, uint32_t r1) {
  asm volatile("stmatrix.sync.aligned.m8n8.x2.trans.shared.b16 [%0], {%1,%2};" ::"r"(a), "r"(r0),
               "r"(r1)
               : "memory");
}

// Round to TF32 (nearest, ties away from zero; see warp_mma.h).  A TF32 value
// is exact as BF16 hi + lo, so split products of rounded operands are TF32
// products.
__device__ __forceinline__ float tf32_round(float x) { return wm::tf32_round(x); }
template <bool TF>
__device__ __forceinline__ float rnd(float x) {
  return TF ? tf32_round(x) : x;
}

// three-way BF16 split of two floats: a = h + m + l exactly (FP32 inputs)
__device__ __forceinline__ void split3(float a, float b, uint32_t& h, uint32_t& m, uint32_t& l) {
  const __nv_bfloat162 hv = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(hv);
  const float ra = a - hf.x, rb = b - hf.y;
  const __nv_bfloat162 mv = __floats2bfloat162_rn(ra, rb);
  const float2 mf = __bfloat1622float2(mv);
  const __nv_bfloat162 lv = __floats2bfloat162_rn(ra - mf.x, rb - mf.y);
  h = *reinterpret_cast<const uint32_t*>(&hv);
  m = *reinterpret_cast<const uint32_t*>(&mv);
  l = *reinterpret_cast<const uint32_t*>(&lv);
}

// GELU and GELU' (gelu_as, gelu_grad_as) come from fno_internal.h.

}  // namespace

// ---------------------------------------------------------------------------
// Kernel parameters and shared-memory plan
// ---------------------------------------------------------------------------
enum { R_U = 0, R_Q, R_X, R_DA, R_STG, R_TB, R_WL, R_BIAS, R_END };

struct EpiM {
  CUtensorMap tmx;     // the 1x1 input as rows [B * Cl][chan], boxes of Cl rows x 128 points
  EpiArgs a;
  int* err;
  const uint2* bz;     // stage-1 B fragments [Nz/4][KZ][2 (hi, lo)][32 lanes]
  long long NxNy, ntiles, chan, plane;
  int Nz, Nt, Jz, Jt, ZB, nzb;
  int NT;              // n-tiles of 8 output channels
  int M1;              // stage-1 m-tiles (two output channels x 8 t modes each)
  int KZ;              // stage-1 k-steps of 16 over (jz, re/im)
  int NZT;             // stage-1 n-tiles of (4 planes x re/im)
  int KL16, KL8;       // stage-3 k-steps over input channels: 16s and an 8 tail
  int MTI, nunits;     // stage 5 (dA mode): m-tiles over Cl + 1 rows; (m, n) units
  int XR, UK, QP;      // x-tile rows; U' row length; Q plane stride (BF16 elements)
  int NX;              // BF16 parts of the x and dA tiles (3 split, 1 plain)
  uint32_t SB, BZO;    // bytes per staging buffer (x tile, then the tile's Bz fragments); Bz offset
  uint32_t off[R_END + 1];
};

constexpr int kXS = kP + 8;  // x / dA row stride (BF16 elements): conflict-free ldmatrix rows

static void epi_mma_geometry(const Dims& d, int mode, int Cs, int Cl, bool split, EpiM& k) {
  k.Nz = (int)d.Nz;
  k.Nt = (int)d.Nt;
  k.Jz = (int)d.Jz;
  k.Jt = (int)d.Jt;
  k.ZB = kP / k.Nt;
  k.nzb = k.Nz / k.ZB;
  k.NT = (Cs + 7) / 8;
  k.M1 = (Cs + 1) / 2;
  k.KZ = (2 * k.Jz + 15) / 16;
  k.NZT = k.ZB / 4;
  const int lin = (mode == EPI_SPECTRAL) ? 0 : Cl;
  k.KL16 = lin / 16;
  k.KL8 = 0;
  if (lin % 16 > 8)
    k.KL16 += 1;
  else if (lin % 16 > 0)
    k.KL8 = 1;
  k.MTI = (mode == EPI_DA) ? (Cl + 1 + 15) / 16 : 0;
  k.nunits = k.MTI * k.NT;
  // stage 5 reads rows 0..16 MTI - 1; rows past Cl only feed discarded dW rows,
  // so rows beyond the tile are clamped to its last row instead of stored
  int xr = 16 * k.KL16 + 8 * k.KL8;
  if (mode == EPI_DA) xr = std::max(xr, (Cl + 1 + 7) / 8 * 8);
  k.XR = xr;
  k.UK = 16 * k.KZ + 8;
  k.QP = 8 * k.NT * 24 + 16;
  k.NX = split ? 3 : 1;
  auto al = [](size_t x) { return (x + 15) / 16 * 16; };
  size_t o = 0;
  k.off[R_U] = (uint32_t)o;  // U' hi, lo: [16 M1][UK]
  o = al(o + 2 * sizeof(uint16_t) * (size_t)(16 * k.M1) * k.UK);
  k.off[R_Q] = (uint32_t)o;  // Q hi, lo: [ZB][QP]
  o = al(o + 2 * sizeof(uint16_t) * (size_t)k.ZB * k.QP);
  k.off[R_X] = (uint32_t)o;  // x tile parts: [NX][XR][kXS]
  o = al(o + sizeof(uint16_t) * (size_t)k.NX * k.XR * kXS);
  k.off[R_DA] = (uint32_t)o;  // dA tile parts (dA mode): [NX][8 NT][kXS]
  if (mode == EPI_DA) o = al(o + sizeof(uint16_t) * (size_t)k.NX * 8 * k.NT * kXS);
  // two staging buffers (128-byte aligned TMA destinations), each the FP32 x
  // tile [Cl][kP] and the tile's Bz fragments
  auto al128 = [](size_t x) { return (x + 127) / 128 * 128; };
  k.BZO = (uint32_t)al128(sizeof(float) * (size_t)lin * kP);
  k.SB = (uint32_t)al128(k.BZO + (size_t)k.NZT * k.KZ * 64 * sizeof(uint2));
  o = al128(o);
  k.off[R_STG] = (uint32_t)o;
  o = al(o + 2 * (size_t)k.SB);
  k.off[R_TB] = (uint32_t)o;  // t-basis A fragments [Nt/16][2][32] uint4
  o = al(o + sizeof(uint4) * 2 * 2 * 32);
  k.off[R_WL] = (uint32_t)o;  // W_lin B fragments [KL16 + KL8][NTM][3][32] uint2
  o = al(o + sizeof(uint2) * (size_t)(k.KL16 + k.KL8) * kNTM * 3 * 32);
  k.off[R_BIAS] = (uint32_t)o;  // bias [8 NTM], two mbarriers, the abort flag
  o = al(o + sizeof(float) * 8 * kNTM + 2 * sizeof(uint64_t) + 16);
  k.off[R_END] = (uint32_t)o;
}

// ---------------------------------------------------------------------------
// Stage-1 B fragments of the inverse z basis, per block of 4 z-planes.  Column
// n = (z, part) of the block: part 0 gives Re, part 1 gives Im of
// sum_jz U[jz] Iz[z][jz]:
//   part 0: B[(jz, 0)] = Re Iz, B[(jz, 1)] = -Im Iz
//   part 1: B[(jz, 0)] = Im Iz, B[(jz, 1)] =  Re Iz
// ---------------------------------------------------------------------------
__global__ void k_epi_mma_bz(const float2* __restrict__ Iz, int Nz, int Jz, int KZ, int tf32,
                             uint2* __restrict__ bz) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int total = (Nz / 4) * KZ * 32;
  if (idx >= total) return;
  const int lane = idx % 32, ks = (idx / 32) % KZ, zq = idx / (32 * KZ);
  const int n = lane / 4, z = 4 * zq + n / 2, part = n % 2;
  auto val = [&](int kk) -> float {
    const int jz = kk / 2, kp = kk % 2;
    if (jz >= Jz) return 0.f;
    const float2 f = Iz[(size_t)z * Jz + jz];
    const float v = (part == 0) ? (kp == 0 ? f.x : -f.y) : (kp == 0 ? f.y : f.x);
    return tf32 ? tf32_round(v) : v;
  };
  const int k0 = 16 * ks + 2 * (lane % 4);
  uint32_t h0, l0, h1, l1;
  split2(val(k0), val(k0 + 1), h0, l0);
  split2(val(k0 + 8), val(k0 + 9), h1, l1);
  const size_t base = (size_t)(zq * KZ + ks) * 2 * 32;
  bz[base + lane] = make_uint2(h0, h1);
  bz[base + 32 + lane] = make_uint2(l0, l1);
}


template <int MODE, bool SPLIT, bool TF>
__global__ void __launch_bounds__(kThreads, 2) k_epi_mma(const __grid_constant__ EpiM k) {
  extern __shared__ __align__(128) unsigned char smem[];
  const EpiArgs& a = k.a;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Cs = a.Cs, Cl = (MODE == EPI_SPECTRAL) ? 0 : a.Cl;
  const int NT = k.NT, Nt = k.Nt, UK = k.UK, QP = k.QP;
  const size_t XP = (size_t)k.XR * kXS;      // stride between x-tile parts
  const size_t DP = (size_t)8 * NT * kXS;    // stride between dA-tile parts

  uint16_t* u_hi = reinterpret_cast<uint16_t*>(smem + k.off[R_U]);
  uint16_t* u_lo = u_hi + (size_t)16 * k.M1 * UK;
  uint16_t* q_hi = reinterpret_cast<uint16_t*>(smem + k.off[R_Q]);
  uint16_t* q_lo = q_hi + (size_t)k.ZB * QP;
  uint16_t* xt = reinterpret_cast<uint16_t*>(smem + k.off[R_X]);
  uint16_t* dt = reinterpret_cast<uint16_t*>(smem + k.off[R_DA]);
  unsigned char* stg = smem + k.off[R_STG];  // buffer q at stg + q * SB
  const uint4* tb = reinterpret_cast<const uint4*>(smem + k.off[R_TB]);
  uint2* wl = reinterpret_cast<uint2*>(smem + k.off[R_WL]);
  float* sb = reinterpret_cast<float*>(smem + k.off[R_BIAS]);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + k.off[R_BIAS] + sizeof(float) * 8 * kNTM);
  volatile int& s_abort = *reinterpret_cast<int*>(bar + 2);

  // TMA destinations must be 128-byte aligned: refuse (uniformly, before any
  // copy is issued) rather than fault if the dynamic shared window is not
  if ((tma::smem_u32(stg) & 127u) != 0u) {
    if (tid == 0 && k.err) atomicExch(k.err, 2);
    return;
  }

  // ---- prologue: zero the operand tiles; constant fragments; bias ----------
  {
    const uint32_t n16 = (k.off[R_STG] - k.off[R_U]) / 16;
    uint4* z4 = reinterpret_cast<uint4*>(smem + k.off[R_U]);
    for (uint32_t e = tid; e < n16; e += kThreads) z4[e] = make_uint4(0, 0, 0, 0);
  }
  if (tid == 0) {
    s_abort = 0;
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::fence_mbar_init();
  }
  // t-basis A fragments Tb[t][k2]: k2 < 8 c/N cos (jt = k2), k2 >= 8 -c/N sin (jt = k2 - 8)
  {
    uint4* tbw = reinterpret_cast<uint4*>(smem + k.off[R_TB]);
    for (int e = tid; e < (Nt / 16) * 32; e += kThreads) {
      const int mt = e / 32, ln = e % 32;
      auto A2 = [&](int t, int k2) -> float {
        const int jt = k2 & 7;
        if (jt >= k.Jt) return 0.f;
        const float2 f = a.It[(size_t)jt * Nt + t];
        return rnd<TF>(k2 < 8 ? f.x : -f.y);
      };
      const int t0 = 16 * mt + ln / 4, c0 = 2 * (ln % 4);
      uint4 h, l;
      split2(A2(t0, c0), A2(t0, c0 + 1), h.x, l.x);
      split2(A2(t0 + 8, c0), A2(t0 + 8, c0 + 1), h.y, l.y);
      split2(A2(t0, c0 + 8), A2(t0, c0 + 9), h.z, l.z);
      split2(A2(t0 + 8, c0 + 8), A2(t0 + 8, c0 + 9), h.w, l.w);
      tbw[(mt * 2 + 0) * 32 + ln] = h;
      tbw[(mt * 2 + 1) * 32 + ln] = l;
    }
  }
  if (MODE != EPI_SPECTRAL) {
    // W_lin B fragments B3[i][o] = W(i, o), three BF16 parts; 16-steps then the 8 tail
    const int nks = k.KL16 + k.KL8;
    for (int e = tid; e < nks * kNTM * 32; e += kThreads) {
      const int ln = e % 32, nt = (e / 32) % kNTM, ks = e / (32 * kNTM);
      const int o = 8 * nt + ln / 4;
      auto W = [&](int i) -> float {
        return (i < Cl && o < Cs) ? rnd<TF>(a.wlin[(size_t)i * a.w_si + (size_t)o * a.w_sc]) : 0.f;
      };
      const int i0 = 16 * ks + 2 * (ln % 4);
      uint2 h, m, l;
      split3(W(i0), W(i0 + 1), h.x, m.x, l.x);
      if (ks < k.KL16)
        split3(W(i0 + 8), W(i0 + 9), h.y, m.y, l.y);
      else
        h.y = m.y = l.y = 0;
      uint2* dst = wl + (size_t)((ks * kNTM + nt) * 3) * 32 + ln;
      dst[0] = h;
      dst[32] = m;
      dst[64] = l;
    }
  }
  for (int o = tid; o < 8 * kNTM; o += kThreads)
    sb[o] = ((MODE == EPI_FWD || MODE == EPI_DA) && o < Cs) ? a.bias[o] : 0.f;
  __syncthreads();
  if (MODE == EPI_DA)  // the row of ones that makes the dW_lin GEMM give db as well
    for (int p = tid; p < kP; p += kThreads) xt[(size_t)Cl * kXS + p] = 0x3f80;  // BF16 1.0

  // ---- tile walk: contiguous range, decoded incrementally ------------------
  const long long t_begin = k.ntiles * blockIdx.x / gridDim.x;
  const long long t_end = k.ntiles * (blockIdx.x + 1) / gridDim.x;
  long long col0 = t_begin / k.nzb;
  int zb = (int)(t_begin - col0 * k.nzb);
  long long b = col0 / k.NxNy, xy = col0 - b * k.NxNy;
  unsigned pending = 0;  // buffers with bulk copies issued and not yet waited for
  // Copies (TMA engine) of a tile's inputs into staging buffer buf, issued by
  // one thread: the x tile (Cl rows x 128 points, one tensor-map box) and the
  // tile's Bz fragments.  Called by every thread (pending is tracked by all).
  const uint32_t bz_bytes = (uint32_t)(k.NZT * k.KZ * 64 * sizeof(uint2));
  auto issue = [&](long long bb, long long xyy, int zbb, int buf) {
    if (tid == 0) {
      unsigned char* dst = stg + (size_t)buf * k.SB;
      tma::fence_proxy_async();
      tma::mbar_arrive_expect_tx(&bar[buf], (uint32_t)(sizeof(float) * Cl * kP) + bz_bytes);
      if (Cl > 0) tma::tma_load_2d(dst, &k.tmx, (int)(xyy * k.plane + (long long)zbb * kP), (int)(bb * Cl), &bar[buf]);
      tma::bulk_g2s(dst + k.BZO, k.bz + (size_t)zbb * k.NZT * k.KZ * 64, bz_bytes, &bar[buf]);
    }
    pending |= 1u << buf;
  };
  if (t_begin < t_end) issue(b, xy, zb, 0);

  uint32_t phase = 0u;  // bit q: the parity the next wait on bar[q] expects
  long long cur_col = -1;
  const int JZT = k.Jz * k.Jt;
  const int zl = (16 * warp) / Nt, t0 = (16 * warp) % Nt;  // this warp's plane and first t
  float ks_sum[2][4], ks_cmp[2][4];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int q = 0; q < 4; ++q) ks_sum[u][q] = ks_cmp[u][q] = 0.f;

  // stage 5 (dA mode): dW_lin and db over the 128 points of the tile whose x
  // and dA tiles are in shared memory, Kahan-folded into this warp's units
  auto stage5 = [&]() {
#pragma unroll
    for (int ui = 0; ui < 2; ++ui) {
      const int u = warp + ui * kWarps;
      if (u < k.nunits) {
        const int mi = u / NT, nt = u - mi * NT;
        // four dependency chains: k-step parity x (large, small) products
        float c5[2][2][4];
#pragma unroll
        for (int x = 0; x < 2; ++x)
#pragma unroll
          for (int y = 0; y < 2; ++y)
#pragma unroll
            for (int q = 0; q < 4; ++q) c5[x][y][q] = 0.f;
        const int row = min(16 * mi + (lane & 7) + 8 * ((lane >> 3) & 1), k.XR - 1);
        const int j = lane >> 3, r = lane & 7;
#pragma unroll 2
        for (int ks = 0; ks < kP / 16; ++ks) {
          float(&cl)[4] = c5[ks & 1][0];
          float(&cs)[4] = c5[ks & 1][1];
          uint32_t ah[4], am[4], al[4];
          const size_t ax = (size_t)row * kXS + 16 * ks + 8 * (lane >> 4);
          const size_t bx = (size_t)(8 * nt + r) * kXS + 16 * ks + 8 * (j & 1);
          ldsm_x4(smem_addr(xt + ax), ah[0], ah[1], ah[2], ah[3]);
          if (SPLIT) {
            ldsm_x4(smem_addr(xt + XP + ax), am[0], am[1], am[2], am[3]);
            ldsm_x4(smem_addr(xt + 2 * XP + ax), al[0], al[1], al[2], al[3]);
            uint2 bh, bm, bl;
            ldsm_x4(smem_addr(dt + ((j >> 1) ? DP : 0) + bx), bh.x, bh.y, bm.x, bm.y);
            ldsm_x2(smem_addr(dt + 2 * DP + bx), bl.x, bl.y);
            mma16(cs, am[0], am[1], am[2], am[3], bm.x, bm.y);
            mma16(cl, am[0], am[1], am[2], am[3], bh.x, bh.y);
            mma16(cs, al[0], al[1], al[2], al[3], bh.x, bh.y);
            mma16(cl, ah[0], ah[1], ah[2], ah[3], bm.x, bm.y);
            mma16(cs, ah[0], ah[1], ah[2], ah[3], bl.x, bl.y);
            mma16(cl, ah[0], ah[1], ah[2], ah[3], bh.x, bh.y);
          } else {
            uint32_t b0, b1;
            ldsm_x2(smem_addr(dt + bx), b0, b1);
            mma16(cl, ah[0], ah[1], ah[2], ah[3], b0, b1);
          }
        }
        float c5s[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          c5s[q] = (c5[0][1][q] + c5[1][1][q]) + (c5[0][0][q] + c5[1][0][q]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float y = c5s[q] - ks_cmp[ui][q];
          const float t = ks_sum[ui][q] + y;
          ks_cmp[ui][q] = (t - ks_sum[ui][q]) - y;
          ks_sum[ui][q] = t;
        }
      }
    }
  };

  bool prev_valid = false;
  for (long long tau = t_begin, c = 0; tau < t_end; ++tau, ++c) {
    const long long tile_ofs = xy * k.plane + (long long)zb * kP;
    const int buf = (int)(c & 1);
    // S0: every shared-memory read of the previous tile is done; the abort
    // decision is the OR over the CTA, so every thread takes the same branch
    if (__syncthreads_or(s_abort != 0)) break;
    // the next tile (prefetch its x tile into the other buffer)
    int zbn = zb + 1;
    long long xyn = xy, bn = b;
    if (zbn == k.nzb) {
      zbn = 0;
      if (++xyn == k.NxNy) {
        xyn = 0;
        ++bn;
      }
    }
    if (tau + 1 < t_end) issue(bn, xyn, zbn, buf ^ 1);
    // a new column: U'[(o, jt)][(jz, re/im)] from the spectrum U[b][o][x][y][jz][jt]
    const long long col = b * k.NxNy + xy;
    const bool newcol = (col != cur_col);
    if (newcol) {
      const float2* U = a.U + ((b * Cs) * k.NxNy + xy) * JZT;
      for (int e = tid; e < Cs * JZT; e += kThreads) {
        const int o = e / JZT, r = e - o * JZT, jz = r / k.Jt, jt = r - jz * k.Jt;
        const float2 u = __ldg(U + (size_t)o * k.NxNy * JZT + r);
        uint32_t h, l;
        split2(rnd<TF>(u.x), rnd<TF>(u.y), h, l);
        const size_t at = (size_t)(o * 8 + jt) * UK + 2 * jz;
        *reinterpret_cast<uint32_t*>(u_hi + at) = h;
        *reinterpret_cast<uint32_t*>(u_lo + at) = l;
      }
      cur_col = col;
    }
    // dA mode: this thread's upstream gradients, in accumulator-fragment order
    float dzr[kNTM][4];
    if (MODE == EPI_DA) {
      const float* dzb = a.dz + (b * Cs + 2 * (lane & 3)) * k.chan + tile_ofs + 16 * warp + (lane >> 2);
      const uint32_t ch = (uint32_t)k.chan;
      const int left = Cs - 2 * (lane & 3);
#pragma unroll
      for (int nt = 0; nt < kNTM; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e)
          dzr[nt][e] = (nt < NT && 8 * nt + (e & 1) < left)
                           ? __ldg(dzb + ((uint32_t)(8 * nt + (e & 1)) * ch + 8 * (e >> 1)))
                           : 0.f;
    }
    // this tile's staging buffer (prefetched during the previous tile)
    if (tma::mbar_wait(&bar[buf], (phase >> buf) & 1u)) {
      phase ^= 1u << buf;
      pending &= ~(1u << buf);
    } else {
      s_abort = 1;
      if (k.err) atomicExch(k.err, 1);
    }
    const unsigned char* sgb = stg + (size_t)buf * k.SB;
    const uint2* bzs = reinterpret_cast<const uint2*>(sgb + k.BZO);
    if (newcol) __syncthreads();  // S1: the rebuilt U' is ready

    // dA mode: stage 5 of the previous tile (its x and dA tiles) beside stage 1
    if (MODE == EPI_DA && prev_valid) stage5();

    // ---- stage 1: inverse z of the tile's planes -> Q (BF16 hi/lo) --------
    // m-tile k goes to warp (k + nunits) % 8, so the warps without a stage-5
    // unit take the m-tiles first; a warp owns m-tiles w1 and w1 + 8
    {
      const int w1 = (warp + kWarps - (k.nunits % kWarps)) % kWarps;
      const bool two = w1 + kWarps < k.M1;
      if (w1 < k.M1) {
        // c1: hi.hi products; c1s: the cross terms (a second dependency chain)
        float c1[2][2][4], c1s[2][2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int n = 0; n < 2; ++n)
#pragma unroll
            for (int q = 0; q < 4; ++q) c1[u][n][q] = c1s[u][n][q] = 0.f;
#pragma unroll
        for (int ks = 0; ks < kKZMax; ++ks) {
          if (ks < k.KZ) {
            uint32_t ah[2][4], al[2][4];
            const int kc = 16 * ks + 8 * (lane >> 4);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              if (u == 0 || two) {
                const int row = 16 * (w1 + u * kWarps) + (lane & 7) + 8 * ((lane >> 3) & 1);
                ldsm_x4(smem_addr(u_hi + (size_t)row * UK + kc), ah[u][0], ah[u][1], ah[u][2], ah[u][3]);
                if (SPLIT)
                  ldsm_x4(smem_addr(u_lo + (size_t)row * UK + kc), al[u][0], al[u][1], al[u][2], al[u][3]);
              }
            }
            uint2 bh[2], bl[2];
#pragma unroll
            for (int ntz = 0; ntz < 2; ++ntz) {
              const uint2* bzp = bzs + (size_t)((ntz < k.NZT ? ntz : 0) * k.KZ + ks) * 64 + lane;
              bh[ntz] = bzp[0];
              bl[ntz] = bzp[32];
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              if (u == 0 || two) {
#pragma unroll
                for (int ntz = 0; ntz < 2; ++ntz) {
                  if (ntz < k.NZT) {
                    if (SPLIT) {
                      mma16(c1s[u][ntz], al[u][0], al[u][1], al[u][2], al[u][3], bh[ntz].x, bh[ntz].y);
                      mma16(c1s[u][ntz], ah[u][0], ah[u][1], ah[u][2], ah[u][3], bl[ntz].x, bl[ntz].y);
                    }
                    mma16(c1[u][ntz], ah[u][0], ah[u][1], ah[u][2], ah[u][3], bh[ntz].x, bh[ntz].y);
                  }
                }
              }
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (u == 0 || two) {
            const int m1 = w1 + u * kWarps;
            float(&cc)[2][4] = c1[u];
#pragma unroll
            for (int n = 0; n < 2; ++n)
#pragma unroll
              for (int q = 0; q < 4; ++q) cc[n][q] += c1s[u][n][q];
            // transposed 8x8 blocks: stored rows are (plane, re/im), columns jt
            const int j = lane >> 3, r = lane & 7;
            const int o = 2 * m1 + (j & 1), ntz = (k.NZT == 2) ? (j >> 1) : 0;
            const size_t at = (size_t)(4 * ntz + (r >> 1)) * QP + (size_t)o * 24 + 8 * (r & 1);
            uint32_t h0, l0, h1, l1;
            split2(rnd<TF>(cc[0][0]), rnd<TF>(cc[0][1]), h0, l0);  // (o_a, planes 0-3)
            split2(rnd<TF>(cc[0][2]), rnd<TF>(cc[0][3]), h1, l1);  // (o_b, planes 0-3)
            if (k.NZT == 2) {
              uint32_t h2, l2, h3, l3;
              split2(rnd<TF>(cc[1][0]), rnd<TF>(cc[1][1]), h2, l2);  // (o_a, planes 4-7)
              split2(rnd<TF>(cc[1][2]), rnd<TF>(cc[1][3]), h3, l3);  // (o_b, planes 4-7)
              stsm_x4_t(smem_addr(q_hi + at), h0, h1, h2, h3);
              stsm_x4_t(smem_addr(q_lo + at), l0, l1, l2, l3);
            } else {
              stsm_x2_t(smem_addr(q_hi + at), h0, h1);
              stsm_x2_t(smem_addr(q_lo + at), l0, l1);
            }
          }
        }
      }
    }

    // dA mode: stage 5 of the previous tile is done with the x tile
    if (MODE == EPI_DA) __syncthreads();
    // ---- the x tile: split into BF16 parts ------------------------------------
    if (Cl > 0) {
      const float* sg = reinterpret_cast<const float*>(sgb);
      for (int e = tid; e < Cl * (kP / 4); e += kThreads) {
        const int i = e / (kP / 4), p4 = 4 * (e % (kP / 4));
        const float4 v = *reinterpret_cast<const float4*>(sg + (size_t)i * kP + p4);
        const size_t at = (size_t)i * kXS + p4;
        if (SPLIT) {
          uint2 h, m, l;
          split3(rnd<TF>(v.x), rnd<TF>(v.y), h.x, m.x, l.x);
          split3(rnd<TF>(v.z), rnd<TF>(v.w), h.y, m.y, l.y);
          *reinterpret_cast<uint2*>(xt + at) = h;
          *reinterpret_cast<uint2*>(xt + XP + at) = m;
          *reinterpret_cast<uint2*>(xt + 2 * XP + at) = l;
        } else {
          uint2 h, l;
          split2(v.x, v.y, h.x, l.x);
          split2(v.z, v.w, h.y, l.y);
          *reinterpret_cast<uint2*>(xt + at) = h;
        }
      }
    }
    __syncthreads();  // S2: Q and the x tile are ready

    // ---- stages 2 + 3: this warp's 16 points, all output channels ----------
    // acc: bias and the hi.hi products; accx: the cross terms of the splits
    // (a second dependency chain, outside the dA mode's register budget)
    constexpr bool XACC = SPLIT && MODE != EPI_DA;
    float acc[kNTM][4], accx[kNTM][4];
#pragma unroll
    for (int nt = 0; nt < kNTM; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) accx[nt][e] = 0.f;
#pragma unroll
    for (int nt = 0; nt < kNTM; ++nt) {
      const float b0 = sb[8 * nt + 2 * (lane & 3)], b1 = sb[8 * nt + 2 * (lane & 3) + 1];
      acc[nt][0] = b0;
      acc[nt][1] = b1;
      acc[nt][2] = b0;
      acc[nt][3] = b1;
    }
    {
      const uint4 h = tb[((t0 >> 4) * 2 + 0) * 32 + lane], l = tb[((t0 >> 4) * 2 + 1) * 32 + lane];
      const uint32_t th[4] = {h.x, h.y, h.z, h.w}, tl[4] = {l.x, l.y, l.z, l.w};
      const int j = lane >> 3, r = lane & 7;
      const uint16_t* qb = (j >> 1) ? q_lo : q_hi;
      uint32_t bq[kNTM][4];
#pragma unroll
      for (int nt = 0; nt < kNTM; ++nt)
        if (nt < NT)
          ldsm_x4(smem_addr(qb + (size_t)zl * QP + (size_t)(8 * nt + r) * 24 + 8 * (j & 1)), bq[nt][0],
                  bq[nt][1], bq[nt][2], bq[nt][3]);
      // product-major over the n-tiles: independent accumulators back to back
      if (SPLIT) {
#pragma unroll
        for (int nt = 0; nt < kNTM; ++nt)
          if (nt < NT) mma16(XACC ? accx[nt] : acc[nt], tl[0], tl[1], tl[2], tl[3], bq[nt][0], bq[nt][1]);
#pragma unroll
        for (int nt = 0; nt < kNTM; ++nt)
          if (nt < NT) mma16(XACC ? accx[nt] : acc[nt], th[0], th[1], th[2], th[3], bq[nt][2], bq[nt][3]);
      }
#pragma unroll
      for (int nt = 0; nt < kNTM; ++nt)
        if (nt < NT) mma16(acc[nt], th[0], th[1], th[2], th[3], bq[nt][0], bq[nt][1]);
    }
    if (MODE != EPI_SPECTRAL) {
      const int j = lane >> 3, r = lane & 7;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        if (ks >= k.KL16) break;
        uint32_t ah[4], am[4], al[4];
        const size_t at = (size_t)(16 * ks + r + 8 * (j >> 1)) * kXS + 16 * warp + 8 * (j & 1);
        ldsm_x4_t(smem_addr(xt + at), ah[0], ah[1], ah[2], ah[3]);
        if (SPLIT) {
          ldsm_x4_t(smem_addr(xt + XP + at), am[0], am[1], am[2], am[3]);
          ldsm_x4_t(smem_addr(xt + 2 * XP + at), al[0], al[1], al[2], al[3]);
        }
        const uint2* wk = wl + (size_t)(ks * kNTM * 3) * 32 + lane;  // [nt][part][lane]
        if (SPLIT) {
          // six products, small terms first, each over all n-tiles back to back
#pragma unroll
          for (int pr = 0; pr < 5; ++pr) {
            const uint32_t* A = (pr == 0 || pr == 3) ? am : (pr == 1 ? al : ah);
            const int bp = (pr == 0 || pr == 4) ? 1 : (pr == 2 ? 2 : 0);
#pragma unroll
            for (int nt = 0; nt < kNTM; ++nt)
              if (nt < NT) {
                const uint2 w = wk[(nt * 3 + bp) * 32];
                mma16(XACC ? accx[nt] : acc[nt], A[0], A[1], A[2], A[3], w.x, w.y);
              }
          }
        }
#pragma unroll
        for (int nt = 0; nt < kNTM; ++nt)
          if (nt < NT) {
            const uint2 w = wk[(nt * 3) * 32];
            mma16(acc[nt], ah[0], ah[1], ah[2], ah[3], w.x, w.y);
          }
      }
      if (k.KL8) {
        const int ks = k.KL16;
        uint32_t ah[2], am[2], al[2];
        const size_t at = (size_t)(16 * ks + r) * kXS + 16 * warp + 8 * (j & 1);
        ldsm_x2_t(smem_addr(xt + at), ah[0], ah[1]);
        if (SPLIT) {
          ldsm_x2_t(smem_addr(xt + XP + at), am[0], am[1]);
          ldsm_x2_t(smem_addr(xt + 2 * XP + at), al[0], al[1]);
        }
        const uint2* wk = wl + (size_t)(ks * kNTM * 3) * 32 + lane;
        if (SPLIT) {
#pragma unroll
          for (int pr = 0; pr < 5; ++pr) {
            const uint32_t* A = (pr == 0 || pr == 3) ? am : (pr == 1 ? al : ah);
            const int bp = (pr == 0 || pr == 4) ? 1 : (pr == 2 ? 2 : 0);
#pragma unroll
            for (int nt = 0; nt < kNTM; ++nt)
              if (nt < NT) mma8(XACC ? accx[nt] : acc[nt], A[0], A[1], wk[(nt * 3 + bp) * 32].x);
          }
        }
#pragma unroll
        for (int nt = 0; nt < kNTM; ++nt)
          if (nt < NT) mma8(acc[nt], ah[0], ah[1], wk[(nt * 3) * 32].x);
      }
    }

    if (XACC) {
#pragma unroll
      for (int nt = 0; nt < kNTM; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[nt][e] += accx[nt][e];
    }
    // ---- pointwise epilogue; stores of 8 consecutive points per channel -----
    {
      const long long oofs = (b * Cs + 2 * (lane & 3)) * k.chan + tile_ofs + 16 * warp + (lane >> 2);
      float* ob = a.out + oofs;
      // training forward: GELU'(A) beside z, from the same erf evaluation
      float* gb = (MODE == EPI_FWD && a.gp) ? a.gp + oofs : nullptr;
      const int ob0 = Cs - 2 * (lane & 3);  // channels left for this lane's column pair
      const uint32_t ch = (uint32_t)k.chan;  // 32 * chan < 2^32 (checked on the host)
#pragma unroll
      for (int nt = 0; nt < kNTM; ++nt) {
        if (nt < NT) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float v = acc[nt][e], g = 0.f;
            if (MODE == EPI_FWD) {
              float phi2, ex;
              phi2_as(v, phi2, ex);
              g = fmaf(v * ex, 0.39894228040143268f, 0.5f * phi2);  // gelu_grad_as(v)
              v = 0.5f * v * phi2;                                  // gelu_as(v)
            }
            if (MODE == EPI_DA) v = dzr[nt][e] * gelu_grad_as(v);
            acc[nt][e] = v;
            if (8 * nt + (e & 1) < ob0) {
              const uint32_t o = (uint32_t)(8 * nt + (e & 1)) * ch + 8 * (e >> 1);
              ob[o] = v;
              if (MODE == EPI_FWD && gb) gb[o] = g;
            }
          }
        }
      }
    }

    if (MODE == EPI_DA) {
      // dA tile [o][p] in BF16 parts for the dW_lin GEMM (transposed 8x8 blocks)
      {
        const int j = (lane >> 3) & 1, r = lane & 7;
#pragma unroll
        for (int nt = 0; nt < kNTM; ++nt) {
          if (nt < NT) {
            const size_t at = (size_t)(8 * nt + r) * kXS + 16 * warp + 8 * j;
            if (SPLIT) {
              uint32_t h0, m0, l0, h1, m1_, l1;
              split3(rnd<TF>(acc[nt][0]), rnd<TF>(acc[nt][1]), h0, m0, l0);
              split3(rnd<TF>(acc[nt][2]), rnd<TF>(acc[nt][3]), h1, m1_, l1);
              stsm_x2_t(smem_addr(dt + at), h0, h1);
              stsm_x2_t(smem_addr(dt + DP + at), m0, m1_);
              stsm_x2_t(smem_addr(dt + 2 * DP + at), l0, l1);
            } else {
              uint32_t h0, l0, h1, l1;
              split2(acc[nt][0], acc[nt][1], h0, l0);
              split2(acc[nt][2], acc[nt][3], h1, l1);
              stsm_x2_t(smem_addr(dt + at), h0, h1);
            }
          }
        }
      }
    }
    prev_valid = true;
    b = bn;
    xy = xyn;
    zb = zbn;
  }
  // dA mode: stage 5 of the last tile (uniform decision, as at S0)
  if (MODE == EPI_DA && prev_valid) {
    if (!__syncthreads_or(s_abort != 0)) stage5();
  }

  // bulk copies still in flight after a timed-out wait must land before exit
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if (pending & (1u << q)) (void)tma::mbar_wait(&bar[q], (phase >> q) & 1u);
  }

  if (MODE == EPI_DA) {
    const int npair = Cl * Cs + Cs;
#pragma unroll
    for (int ui = 0; ui < 2; ++ui) {
      const int u = warp + ui * kWarps;
      if (u < k.nunits) {
        const int mi = u / NT, nt = u - mi * NT;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = 16 * mi + (lane >> 2) + 8 * (q >> 1);
          const int o = 8 * nt + 2 * (lane & 3) + (q & 1);
          const float v = ks_sum[ui][q] - ks_cmp[ui][q];
          if (o < Cs && i <= Cl) {
            const int idx = (i < Cl) ? i * Cs + o : Cl * Cs + o;
            a.part[(long long)blockIdx.x * npair + idx] = v;
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
size_t epilogue_mma_table_bytes(const Dims& d) {
  const int KZ = (int)((2 * d.Jz + 15) / 16);
  return sizeof(uint2) * (size_t)((d.Nz + 3) / 4) * KZ * 2 * 32;
}

bool epilogue_mma_supported(const Dims& d, int mode, int Cs, int Cl, char* why, size_t nwhy) {
  auto no = [&](const char* m) {
    if (why && nwhy) snprintf(why, nwhy, "%s", m);
    return false;
  };
  if (d.Nt != 16 && d.Nt != 32) return no("mma epilogue needs Nt of 16 or 32");
  if (d.Jt > 8) return no("mma epilogue needs mt <= 8");
  if (d.Nz % (kP / d.Nt) != 0) return no("mma epilogue needs Nz a multiple of 128 / Nt");
  if (d.Jz > 24) return no("mma epilogue needs 2*mz <= 24");
  if ((long long)d.Nx * d.Ny * d.Nz * d.Nt * 32 >= (1LL << 32))
    return no("mma epilogue needs 32 * Nx*Ny*Nz*Nt < 2^32");
  if (Cs < 1 || Cs > 8 * kNTM) return no("mma epilogue needs 1..32 output channels");
  if (mode != EPI_SPECTRAL && (Cl < 1 || Cl > kClMax)) return no("mma epilogue needs 1..32 1x1 inputs");
  EpiM k{};
  epi_mma_geometry(d, mode, Cs, Cl, true, k);
  if (mode == EPI_DA && k.nunits > 2 * kWarps) return no("mma epilogue: too many dW_lin tiles");
  if (k.off[R_END] > 227 * 1024) return no("mma epilogue: shared memory");
  return true;
}

template <int MODE, bool SPLIT, bool TF>
static cudaError_t launch_mma_t(const EpiM& k, int* grid_used, cudaStream_t s) {
  const void* kern = (const void*)k_epi_mma<MODE, SPLIT, TF>;
  const size_t smem = k.off[R_END];
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  long long g = (long long)per_sm * sm_count();
  if (g > k.ntiles) g = k.ntiles;
  if (g > epilogue_max_grid()) g = epilogue_max_grid();
  if (g < 1) g = 1;
  if (grid_used) *grid_used = (int)g;
  static const char* names[3][4] = {
      {"fno_epi_spectral_mma_bf16", "fno_epi_fwd_mma_bf16", "fno_epi_da_mma_bf16", "fno_epi_dx_mma_bf16"},
      {"fno_epi_spectral_mma_bf16x3", "fno_epi_fwd_mma_bf16x3", "fno_epi_da_mma_bf16x3",
       "fno_epi_dx_mma_bf16x3"},
      {"fno_epi_spectral_mma_tf32", "fno_epi_fwd_mma_tf32", "fno_epi_da_mma_tf32", "fno_epi_dx_mma_tf32"}};
  // the forward of a training step also stores GELU'(A): its own name, so that
  // timings and byte counts tell the two apart
  static const char* train_names[3] = {"fno_epi_fwd_train_mma_bf16", "fno_epi_fwd_train_mma_bf16x3",
                                       "fno_epi_fwd_train_mma_tf32"};
  const int pv = TF ? 2 : (SPLIT ? 1 : 0);
  const char* name = (MODE == EPI_FWD && k.a.gp) ? train_names[pv] : names[pv][MODE];
  FNO_LAUNCH(name, (k_epi_mma<MODE, SPLIT, TF>), (int)g, kThreads, smem, s, k);
  return cudaSuccess;
}

template <int MODE>
static cudaError_t launch_mma_m(const EpiM& k, bool split, bool tf32, int* g, cudaStream_t s) {
  if (tf32) return launch_mma_t<MODE, true, true>(k, g, s);
  return split ? launch_mma_t<MODE, true, false>(k, g, s) : launch_mma_t<MODE, false, false>(k, g, s);
}

// Tiled tensor map of an FP32 array, encoded through the driver entry point
// (no link-time driver dependency).  strides: bytes of dimensions 1 .. rank-1.
cudaError_t encode_tiled(CUtensorMap* map, const void* base, int rank, const cuuint64_t* dims,
                         const cuuint64_t* strides, const cuuint32_t* box, bool swizzle128) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                CUtensorMapFloatOOBfill);
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return cudaErrorNotSupported;
    fn = reinterpret_cast<EncodeFn>(p);
  }
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor map of a [rows][chan] FP32 array with boxes of box_rows x 128 points.
cudaError_t encode_x_map(CUtensorMap* map, const float* base, long long chan, long long rows,
                         int box_rows) {
  const cuuint64_t dims[2] = {(cuuint64_t)chan, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)chan * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kP, (cuuint32_t)box_rows};
  return encode_tiled(map, base, 2, dims, strides, box, false);
}

cudaError_t launch_epilogue_mma(const Dims& d, const EpiArgs& a, bool split, bool tf32, void* table,
                                int* err, int* grid_used, cudaStream_t s) {
  EpiM k{};
  k.a = a;
  k.err = err;
  epi_mma_geometry(d, a.mode, a.Cs, a.Cl, split, k);
  k.NxNy = d.Nx * d.Ny;
  k.plane = d.Nz * d.Nt;
  k.chan = k.NxNy * k.plane;
  k.ntiles = d.B * k.NxNy * (long long)k.nzb;
  uint2* bz = static_cast<uint2*>(table);
  k.bz = bz;
  if (a.mode != EPI_SPECTRAL) {
    cudaError_t e = encode_x_map(&k.tmx, a.lin_in, k.chan, d.B * (long long)a.Cl, a.Cl);
    if (e != cudaSuccess) return e;
  }
  {
    const int total = (k.Nz / 4) * k.KZ * 32;
    FNO_LAUNCH("fno_epi_mma_tables", k_epi_mma_bz, (total + 255) / 256, 256, 0, s, a.Iz, k.Nz,
               k.Jz, k.KZ, tf32 ? 1 : 0, bz);
  }
  switch (a.mode) {
    case EPI_SPECTRAL: return launch_mma_m<EPI_SPECTRAL>(k, split, tf32, grid_used, s);
    case EPI_FWD: return launch_mma_m<EPI_FWD>(k, split, tf32, grid_used, s);
    case EPI_DA: return launch_mma_m<EPI_DA>(k, split, tf32, grid_used, s);
    default: return launch_mma_m<EPI_DX>(k, split, tf32, grid_used, s);
  }
}

}  // namespace fno

namespace fno {

// ---------------------------------------------------------------------------
// One complex DFT axis on the tensor cores (the y and x stages of Alg. 2, both
// directions):  out[o][q][i] = sum_n T[q][n] in[o][n][i]   (complex).
// As a real GEMM per o: rows m = 2q + (re, im) of the output, k = 2n + (re, im)
// of the input, columns i:
//   A[(q,0)][(n,0)] = Re T, A[(q,0)][(n,1)] = -Im T, A[(q,1)][(n,0)] = Im T,
//   A[(q,1)][(n,1)] = Re T;  B[(n, part)][i] = part of in[o][n][i].
// A B-fragment slot pair (2 t4, 2 t4 + 1) is exactly one input float2.  Each
// warp computes 16 columns of one o; with few m-tiles (M <= 64) it streams K,
// otherwise it holds all of K for its columns and walks the m-tiles.  Its
// loads run one k-step (streaming) or one task (walk) ahead of the products,
// so that their latency overlaps tensor-core work.  Split BF16 uses three-way
// splits of both operands (six products), BF16 one product.
// ---------------------------------------------------------------------------
struct LineM {
  const float2* in;
  float2* out;
  const float2* tab;  // [nout][nin]
  long long outer, inner, ncb;  // ncb: 16-column blocks per o
  int nin, nout, MT, KS;
};

constexpr int kLineMTMax = 4;  // m-tiles held at once when streaming K
constexpr int kLineKSMax = 4;  // k-steps held at once when walking m-tiles

template <bool SPLIT, bool KOUTER, bool TF>
__global__ void __launch_bounds__(256) k_line_mma(const LineM L) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint4* af = reinterpret_cast<uint4*>(smem);  // [MT][KS][parts][32 lanes]
  constexpr int NP = SPLIT ? 3 : 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g8 = lane >> 2, t4 = lane & 3;
  const int MT = L.MT, KS = L.KS, nin = L.nin, nout = L.nout;

  // ---- A fragments of the basis, once per CTA ----------------------------
  for (int e = tid; e < MT * KS * 32; e += 256) {
    const int ln = e % 32, ks = (e / 32) % KS, mt = e / (32 * KS);
    auto A = [&](int m, int kk) -> float {
      const int q = m >> 1, po = m & 1, n = kk >> 1, pi = kk & 1;
      if (q >= nout || n >= nin) return 0.f;
      const float2 t = L.tab[(size_t)q * nin + n];
      return rnd<TF>((po == 0) ? (pi == 0 ? t.x : -t.y) : (pi == 0 ? t.y : t.x));
    };
    const int r0 = 16 * mt + ln / 4, c0 = 16 * ks + 2 * (ln % 4);
    uint4 h, m, l;
    split3(A(r0, c0), A(r0, c0 + 1), h.x, m.x, l.x);
    split3(A(r0 + 8, c0), A(r0 + 8, c0 + 1), h.y, m.y, l.y);
    split3(A(r0, c0 + 8), A(r0, c0 + 9), h.z, m.z, l.z);
    split3(A(r0 + 8, c0 + 8), A(r0 + 8, c0 + 9), h.w, m.w, l.w);
    uint4* dst = af + ((size_t)(mt * KS + ks) * NP) * 32 + ln;
    dst[0] = h;
    if (SPLIT) {
      dst[32] = m;
      dst[64] = l;
    }
  }
  __syncthreads();

  const long long ntask = L.outer * L.ncb;
  const long long nw = (long long)gridDim.x * 8;
  // B inputs of k-step ks for the 16 columns from i0 (rows n = 8 ks + 4 hf + t4 of src)
  auto loadRaw = [&](const float2* src, long long i0, int ks, float2 (&vr)[2][2]) {
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const long long col = i0 + 8 * nt + g8;
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        const int n = 8 * ks + 4 * hf + t4;
        vr[nt][hf] = make_float2(0.f, 0.f);
        if (n < nin && col < L.inner) vr[nt][hf] = __ldg(src + (size_t)n * L.inner + col);
      }
    }
  };
  // every k-step's inputs of task tk (the m-tile walk holds them all)
  auto loadTask = [&](long long tk, float2 (&v)[kLineKSMax][2][2]) {
    const long long o = tk / L.ncb;
    const float2* src = L.in + (size_t)o * nin * L.inner;
#pragma unroll
    for (int ks = 0; ks < kLineKSMax; ++ks)
      if (ks < KS) loadRaw(src, (tk - o * L.ncb) * 16, ks, v[ks]);
  };
  // m-tile walk: the next task's inputs are in flight while this task's products run
  float2 vnx[kLineKSMax][2][2];
  if (!KOUTER && (long long)blockIdx.x * 8 + warp < ntask) loadTask((long long)blockIdx.x * 8 + warp, vnx);
  for (long long task = (long long)blockIdx.x * 8 + warp; task < ntask; task += nw) {
    const long long o = task / L.ncb;
    const long long i0 = (task - o * L.ncb) * 16;
    const float2* src = L.in + (size_t)o * nin * L.inner;
    float2* dst = L.out + (size_t)o * nout * L.inner;
    // B fragments (split parts) of one k-step for the two n-tiles of this warp's 16 columns
    auto convB = [&](const float2 (&vr)[2][2], uint32_t (&bh)[2][2], uint32_t (&bm)[2][2], uint32_t (&bl)[2][2]) {
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          float2 v = vr[nt][hf];
          v.x = rnd<TF>(v.x);
          v.y = rnd<TF>(v.y);
          if (SPLIT)
            split3(v.x, v.y, bh[nt][hf], bm[nt][hf], bl[nt][hf]);
          else {
            uint32_t lo;
            split2(v.x, v.y, bh[nt][hf], lo);
          }
        }
      }
    };
    // C fragment of m-tile mt, n-tile nt -> out (re on even rows, im on odd rows)
    auto store = [&](int mt, int nt, const float (&c)[4]) {
      const float p0 = __shfl_xor_sync(0xffffffffu, c[0], 4), p1 = __shfl_xor_sync(0xffffffffu, c[1], 4);
      const float p2 = __shfl_xor_sync(0xffffffffu, c[2], 4), p3 = __shfl_xor_sync(0xffffffffu, c[3], 4);
      const bool even = (g8 & 1) == 0;
      // even rows g: (q, re) and (q + 4, re); the partner lane holds the im parts
      const int q = (16 * mt + (g8 & ~1)) / 2 + (even ? 0 : 4);
      const float4 v = even ? make_float4(c[0], p0, c[1], p1) : make_float4(p2, c[2], p3, c[3]);
      const long long col = i0 + 8 * nt + 2 * t4;
      if (q < nout && col + 1 < L.inner && (L.inner & 1) == 0)
        *reinterpret_cast<float4*>(dst + (size_t)q * L.inner + col) = v;
      else if (q < nout) {
        if (col < L.inner) dst[(size_t)q * L.inner + col] = make_float2(v.x, v.y);
        if (col + 1 < L.inner) dst[(size_t)q * L.inner + col + 1] = make_float2(v.z, v.w);
      }
    };
    auto mma_parts = [&](float (&d)[4], const uint4* a, const uint32_t (&bh)[2], const uint32_t (&bm)[2],
                         const uint32_t (&bl)[2]) {
      const uint4 ah = a[0];
      if (SPLIT) {
        const uint4 am = a[32], al = a[64];
        mma16(d, am.x, am.y, am.z, am.w, bm[0], bm[1]);
        mma16(d, al.x, al.y, al.z, al.w, bh[0], bh[1]);
        mma16(d, ah.x, ah.y, ah.z, ah.w, bl[0], bl[1]);
        mma16(d, am.x, am.y, am.z, am.w, bh[0], bh[1]);
        mma16(d, ah.x, ah.y, ah.z, ah.w, bm[0], bm[1]);
      }
      mma16(d, ah.x, ah.y, ah.z, ah.w, bh[0], bh[1]);
    };
    if (KOUTER) {
      // few m-tiles: stream K, all m-tiles and both n-tiles in registers
      float acc[kLineMTMax][2][4];
#pragma unroll
      for (int mt = 0; mt < kLineMTMax; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.f;
      // the tensor-core FP32 accumulation is not round-to-nearest, so each
      // k-step accumulates from zero and is added into the total in FP32; the
      // next k-step's inputs are loaded before this k-step's products
      float2 vr[2][2];
      loadRaw(src, i0, 0, vr);
      for (int ks = 0; ks < KS; ++ks) {
        uint32_t bh[2][2], bm[2][2], bl[2][2];
        convB(vr, bh, bm, bl);
        if (ks + 1 < KS) loadRaw(src, i0, ks + 1, vr);
#pragma unroll
        for (int mt = 0; mt < kLineMTMax; ++mt)
          if (mt < MT) {
            const uint4* a = af + ((size_t)(mt * KS + ks) * NP) * 32 + lane;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
              float part[4] = {0.f, 0.f, 0.f, 0.f};
              mma_parts(part, a, bh[nt], bm[nt], bl[nt]);
#pragma unroll
              for (int q = 0; q < 4; ++q) acc[mt][nt][q] += part[q];
            }
          }
      }
#pragma unroll
      for (int mt = 0; mt < kLineMTMax; ++mt)
        if (mt < MT)
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) store(mt, nt, acc[mt][nt]);
    } else {
      // few k-steps: every B fragment of the columns in registers, walk the m-tiles
      uint32_t bh[kLineKSMax][2][2], bm[kLineKSMax][2][2], bl[kLineKSMax][2][2];
#pragma unroll
      for (int ks = 0; ks < kLineKSMax; ++ks)
        if (ks < KS) convB(vnx[ks], bh[ks], bm[ks], bl[ks]);
      if (task + nw < ntask) loadTask(task + nw, vnx);
      for (int mt = 0; mt < MT; ++mt) {
        float acc[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[nt][q] = 0.f;
#pragma unroll
        for (int ks = 0; ks < kLineKSMax; ++ks)
          if (ks < KS) {
            const uint4* a = af + ((size_t)(mt * KS + ks) * NP) * 32 + lane;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
              float part[4] = {0.f, 0.f, 0.f, 0.f};
              mma_parts(part, a, bh[ks][nt], bm[ks][nt], bl[ks][nt]);
#pragma unroll
              for (int q = 0; q < 4; ++q) acc[nt][q] += part[q];
            }
          }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) store(mt, nt, acc[nt]);
      }
    }
  }
}

bool line_mma_supported(int nin, int nout) {
  const int MT = (2 * nout + 15) / 16, KS = (2 * nin + 15) / 16;
  return MT <= kLineMTMax || KS <= kLineKSMax;
}

template <bool SPLIT, bool KOUTER, bool TF>
static cudaError_t launch_line_t(const LineM& L, size_t smem, const char* name, cudaStream_t s) {
  const void* kern = (const void*)k_line_mma<SPLIT, KOUTER, TF>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const long long tasks = L.outer * L.ncb;
  long long g = (long long)per_sm * sm_count();
  if (g * 8 > tasks) g = (tasks + 7) / 8;
  if (g < 1) g = 1;
  FNO_LAUNCH(name, (k_line_mma<SPLIT, KOUTER, TF>), (int)g, 256, smem, s, L);
  return cudaSuccess;
}

cudaError_t launch_line_mma(const float2* in, float2* out, int64_t outer, int nin, int nout,
                            int64_t inner, const float2* tab, bool split, bool tf32, cudaStream_t s) {
  if (outer <= 0 || inner <= 0) return cudaSuccess;
  LineM L{};
  L.in = in;
  L.out = out;
  L.tab = tab;
  L.outer = outer;
  L.inner = inner;
  L.ncb = (inner + 15) / 16;
  L.nin = nin;
  L.nout = nout;
  L.MT = (2 * nout + 15) / 16;
  L.KS = (2 * nin + 15) / 16;
  const bool kouter = L.MT <= kLineMTMax;
  if (!kouter && L.KS > kLineKSMax) return cudaErrorInvalidValue;
  split = split || tf32;
  const size_t smem = sizeof(uint4) * (size_t)L.MT * L.KS * (split ? 3 : 1) * 32;
  if (tf32)
    return kouter ? launch_line_t<true, true, true>(L, smem, "fno_line_mma_tf32", s)
                  : launch_line_t<true, false, true>(L, smem, "fno_line_mma_tf32", s);
  if (split)
    return kouter ? launch_line_t<true, true, false>(L, smem, "fno_line_mma_bf16x3", s)
                  : launch_line_t<true, false, false>(L, smem, "fno_line_mma_bf16x3", s);
  return kouter ? launch_line_t<false, true, false>(L, smem, "fno_line_mma_bf16", s)
                : launch_line_t<false, false, false>(L, smem, "fno_line_mma_bf16", s);
}

// ---------------------------------------------------------------------------
// Inverse t stage to real points on the tensor cores, for grids whose Nt the
// fused epilogues do not tile (Nt other than 16 and 32, e.g. the paper's 84
// and 86):
//   S[r][t] = sum_jt Re(It[jt][t] V[r][jt])        r = (column, z), t < Nt
// with It carrying c(kt)/N.  As a real GEMM over K = 16 = (jt, re/im):
//   A[r][(jt, 0)] = Re V, A[r][(jt, 1)] = Im V   (one float2 of V fills one
//   A-fragment slot pair), B[(jt, 0)][t] = Re It, B[(jt, 1)][t] = -Im It.
// A warp owns 16 rows at a time, loads the next 16 before this one's products
// and walks the n-tiles of 8 t into a shared-memory tile of its own; the 16
// rows are one contiguous run of out, which the warp then writes (or adds to:
// the dX form, whose 1x1 term is written first) with 16-byte accesses.  Split
// BF16 and TF32 take three-way splits of both operands (six products), BF16 one.
// ---------------------------------------------------------------------------
struct SynthT {
  const float2* V;   // [R][Jt]
  const float2* It;  // [Jt][Nt]
  float* out;        // [R][Nt]
  long long R;
  int Nt, Jt, NTN, accumulate;
};

constexpr int kSynthNTMax = 16;  // n-tiles of 8 t (Nt <= 128)

template <bool SPLIT, bool TF>
__global__ void __launch_bounds__(256) k_synth_t(const SynthT k) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int NP = SPLIT ? 3 : 1;
  uint2* bfr = reinterpret_cast<uint2*>(smem);  // [NTN][NP][32 lanes]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g8 = lane >> 2, t4 = lane & 3;
  const int Nt = k.Nt, Jt = k.Jt;

  // B fragments of the t basis: b0 = (k 2 t4, 2 t4 + 1; n g8) = jt t4,
  // b1 = the same at jt t4 + 4; n = t
  for (int e = tid; e < k.NTN * 32; e += 256) {
    const int nt = e >> 5, ln = e & 31;
    const int t = 8 * nt + (ln >> 2);
    uint32_t h[2], m[2], l[2];
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      const int jt = (ln & 3) + 4 * hf;
      float re = 0.f, im = 0.f;
      if (jt < Jt && t < Nt) {
        const float2 f = k.It[(size_t)jt * Nt + t];
        re = rnd<TF>(f.x);
        im = rnd<TF>(-f.y);
      }
      if (SPLIT)
        split3(re, im, h[hf], m[hf], l[hf]);
      else
        split2(re, im, h[hf], l[hf]);
    }
    uint2* dst = bfr + (size_t)nt * NP * 32 + ln;
    dst[0] = make_uint2(h[0], h[1]);
    if (SPLIT) {
      dst[32] = make_uint2(m[0], m[1]);
      dst[64] = make_uint2(l[0], l[1]);
    }
  }
  __syncthreads();

  const long long nmt = (k.R + 15) / 16;
  const long long nw = (long long)gridDim.x * 8;
  // A inputs of m-tile mt: v[q] = V[16 mt + g8 + 8 (q & 1)][t4 + 4 (q >> 1)]
  auto loadA = [&](long long mt, float2 (&v)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long r = 16 * mt + g8 + 8 * (q & 1);
      const int jt = t4 + 4 * (q >> 1);
      v[q] = make_float2(0.f, 0.f);
      if (r < k.R && jt < Jt) v[q] = __ldg(k.V + (size_t)r * Jt + jt);
    }
  };
  // this warp's output tile [16 rows][LD]; columns past Nt are never copied out
  const int LD = 8 * k.NTN + 4;
  float* tile = reinterpret_cast<float*>(smem + sizeof(uint2) * (size_t)k.NTN * NP * 32) + warp * 16 * LD;
  const bool out16 = ((reinterpret_cast<uintptr_t>(k.out) & 15u) == 0);
  float2 vn[4];
  long long mt = (long long)blockIdx.x * 8 + warp;
  if (mt < nmt) loadA(mt, vn);
  for (; mt < nmt; mt += nw) {
    uint32_t ah[4], am[4], al[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float x = rnd<TF>(vn[q].x), y = rnd<TF>(vn[q].y);
      if (SPLIT)
        split3(x, y, ah[q], am[q], al[q]);
      else
        split2(x, y, ah[q], al[q]);
    }
    if (mt + nw < nmt) loadA(mt + nw, vn);
    for (int nt = 0; nt < k.NTN; ++nt) {
      const uint2* b = bfr + (size_t)nt * NP * 32 + lane;
      const uint2 bh = b[0];
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      if (SPLIT) {
        const uint2 bm = b[32], bl = b[64];
        mma16(c, am[0], am[1], am[2], am[3], bm.x, bm.y);
        mma16(c, al[0], al[1], al[2], al[3], bh.x, bh.y);
        mma16(c, ah[0], ah[1], ah[2], ah[3], bl.x, bl.y);
        mma16(c, am[0], am[1], am[2], am[3], bh.x, bh.y);
        mma16(c, ah[0], ah[1], ah[2], ah[3], bm.x, bm.y);
      }
      mma16(c, ah[0], ah[1], ah[2], ah[3], bh.x, bh.y);
      // c0, c1: row g8, t = 8 nt + 2 t4 (+1); c2, c3: row g8 + 8
      const int t = 8 * nt + 2 * t4;
      *reinterpret_cast<float2*>(tile + g8 * LD + t) = make_float2(c[0], c[1]);
      *reinterpret_cast<float2*>(tile + (g8 + 8) * LD + t) = make_float2(c[2], c[3]);
    }
    __syncwarp();
    // rows 16 mt .. 16 mt + nrow - 1 are out[16 mt Nt, (16 mt + nrow) Nt)
    const long long rb = 16 * mt;
    const int nrow = (int)min(16LL, k.R - rb);
    const int cnt = nrow * Nt;
    float* o = k.out + (size_t)rb * Nt;
    auto at = [&](int e) -> float {
      const int row = e / Nt;
      return tile[row * LD + (e - row * Nt)];
    };
    if (out16 && (cnt & 3) == 0 && ((rb * Nt) & 3) == 0) {
      float4* o4 = reinterpret_cast<float4*>(o);
      for (int e4 = lane; e4 < cnt / 4; e4 += 32) {
        float4 v = make_float4(at(4 * e4), at(4 * e4 + 1), at(4 * e4 + 2), at(4 * e4 + 3));
        if (k.accumulate) {
          const float4 c = o4[e4];
          v.x += c.x;
          v.y += c.y;
          v.z += c.z;
          v.w += c.w;
        }
        o4[e4] = v;
      }
    } else {
      for (int e = lane; e < cnt; e += 32) o[e] = k.accumulate ? o[e] + at(e) : at(e);
    }
    __syncwarp();
  }
}

bool synth_t_supported(int Nt, int Jt) { return Nt >= 1 && Nt <= 8 * kSynthNTMax && Jt >= 1 && Jt <= 8; }

template <bool SPLIT, bool TF>
static cudaError_t launch_synth_k(const SynthT& k, size_t smem, const char* name, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_synth_t<SPLIT, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_synth_t<SPLIT, TF>, 256, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const long long tiles = (k.R + 15) / 16;
  long long g = (long long)per_sm * sm_count();
  if (g * 8 > tiles) g = (tiles + 7) / 8;
  if (g < 1) g = 1;
  FNO_LAUNCH(name, (k_synth_t<SPLIT, TF>), (int)g, 256, smem, s, k);
  return cudaSuccess;
}

cudaError_t launch_synth_t(const float2* V, float* out, int64_t R, int Nt, int Jt, const float2* It,
                           bool accumulate, bool split, bool tf32, cudaStream_t s) {
  if (R <= 0) return cudaSuccess;
  if (!synth_t_supported(Nt, Jt)) return cudaErrorInvalidValue;
  SynthT k{};
  k.V = V;
  k.It = It;
  k.out = out;
  k.R = R;
  k.Nt = Nt;
  k.Jt = Jt;
  k.NTN = (Nt + 7) / 8;
  k.accumulate = accumulate ? 1 : 0;
  split = split || tf32;
  // basis fragments (at most 12 KB) and eight warp tiles of 16 x (8 NTN + 4) floats (at most 66 KB)
  const size_t smem = sizeof(uint2) * (size_t)k.NTN * (split ? 3 : 1) * 32 +
                      sizeof(float) * 8 * 16 * (size_t)(8 * k.NTN + 4);
  if (tf32) return launch_synth_k<true, true>(k, smem, "fno_synth_t_tf32", s);
  if (split) return launch_synth_k<true, false>(k, smem, "fno_synth_t_bf16x3", s);
  return launch_synth_k<false, false>(k, smem, "fno_synth_t_bf16", s);
}

}  // namespace fno

// ============================================================================
// Forward pruned DFT over t then z of every (b, c, x, y) column, both stages on
// mma.sync in registers (the first half of F_yzt, S_yzt in Alg. 2).
//
//   t stage  P_ri[jt][z] = sum_t F_ri[jt][t] X[z][t]        ri = re (cos), im (-sin)
//   z stage  T[kz][jt]   = sum_z Fz[kz][z] (P_re + i P_im)[jt][z]
//            Re T = Fz_r P_re - Fz_i P_im,   Im T = Fz_r P_im + Fz_i P_re
//
// One warp owns one column at a time.  The t stage is m16n8k16 with the basis
// as the A operand (rows ri * 8 + jt) and the column as B (k = t, n = z): its C
// fragments of the n-tiles 2 ks and 2 ks + 1 hold (jt = lane / 4, z = 16 ks +
// 2 (lane % 4) + {0, 1} and + 8), which is exactly the B fragment (k = z, n =
// jt) of the z stage's k-step ks -- the two stages chain in registers, with no
// shared-memory round trip and no TMEM.  The t stage's k slots map to four
// consecutive t per thread (one float4 of the staged column; the basis
// fragments use the same map).  The z basis sits in shared memory already in
// A-fragment order (one 16-byte load per lane and operand part).  Each z
// k-step accumulates from zero and is added into FP32 totals, so tensor-core
// accumulation chains stay at six MMAs.
//
// Columns arrive by bulk copy (TMA engine) into a ring of S stages (16 KB: G
// columns, or one column in NCH chunks); warp 0 is the producer, warps
// 1..kTzWarps take the column units w - 1, w - 1 + kTzWarps, ... in order, so a
// consumer skips stages: it waits on a stage's barrier only after the producer
// has published that it issued the stage (see `issued`).  Two CTAs share an SM
// (two producers measured 1.24 ms against 1.47 ms for one at 128^3 x 32; larger
// or smaller stages were slower).  Every wait is bounded: on timeout the kernel
// raises *err, the producer waits (bounded) for its copies in flight, and all
// warps return.
// ============================================================================
namespace fno {
namespace {

constexpr int kTzWarps = 8;                      // consumer warps
constexpr int kTzThreads = 32 * (kTzWarps + 1);
constexpr int kTzKTMax = 8;                      // t-stage k-steps (Nt <= 128)
constexpr long long kTzWait = 4000000000LL;      // about 2 s of SM clocks

struct TzM {
  const float* in;     // [ncol][Nz][Nt]
  float2* out;         // [ncol][Jz][Jt]
  const float2* Ft;    // [Jt][Nt]  (cos, -sin) * scale
  const float2* Fz;    // [Jz][Nz]  (cos, -sin)
  int* err;
  long long ncol, nunits;   // units: G whole columns, or one column in NCH chunks
  int Nz, Nt, Jz, Jt, KT, KZ, G, S, NCH, zc;   // chunks of zc rows (the last may be shorter)
  uint32_t col_floats, o_fz, o_ft, o_ring, stage_bytes, o_bar;
};

// Wait (bounded) until the producer has issued stage g; false on timeout or abort.
__device__ __forceinline__ bool tz_wait_issued(volatile int* issued, volatile int* abort_flag,
                                               int g) {
  if (*issued > g) return true;
  const long long t0 = clock64();
  while (*issued <= g) {
    if (*abort_flag || clock64() - t0 > kTzWait) return false;
    __nanosleep(64);
  }
  return true;
}

// CTAs per SM: two producers per SM measured faster than one; four z m-tiles
// need the registers of a whole SM.
__host__ __device__ constexpr int tz_ctas(int mz) { return mz <= 2 ? 2 : 1; }

// KTR > 0: the t basis fragments live in registers for up to KTR k-steps (Nt <=
// 16 KTR); KTR = 0: they are read from a shared-memory table (longer Nt).
template <int MZ, int KTR, bool SPLIT, bool TF>
__global__ void __launch_bounds__(kTzThreads, tz_ctas(MZ)) k_fwd_tz_mma(const __grid_constant__ TzM p) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g8 = lane >> 2, t4 = lane & 3;
  const int S = p.S;
  uint4* fzf = reinterpret_cast<uint4*>(sm + p.o_fz);  // [MZ][KZ][4 parts][32 lanes]
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + p.o_bar);
  uint64_t* empty = full + S;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + S);
  // stages issued so far: a consumer waits on stage g's barrier only once the
  // producer has issued g.  Issuing g needed stage g - S consumed (so landed),
  // so the slot's barrier is then exactly in stage g's phase and the parity
  // test cannot match an older, still open phase.
  volatile int* issued = abort_flag + 1;

  // z basis in A-fragment order: parts (re hi, re lo, im hi, im lo); rows kz,
  // cols z; a0 = (kz g8, z 2 t4 + {0,1}), a1 = (kz g8 + 8, ...), a2, a3 at z + 8
  for (int e = tid; e < MZ * p.KZ * 32; e += kTzThreads) {
    const int ln = e & 31, ks = (e >> 5) % p.KZ, mt = (e >> 5) / p.KZ;
    const int r0 = 16 * mt + (ln >> 2), c0 = 16 * ks + 2 * (ln & 3);
    auto F = [&](int kz, int z, int im) -> float {
      if (kz >= p.Jz || z >= p.Nz) return 0.f;
      const float2 f = p.Fz[(long long)kz * p.Nz + z];
      return rnd<TF>(im ? f.y : f.x);
    };
#pragma unroll
    for (int im = 0; im < 2; ++im) {
      uint32_t h[4], l[4];
      split2(F(r0, c0, im), F(r0, c0 + 1, im), h[0], l[0]);
      split2(F(r0 + 8, c0, im), F(r0 + 8, c0 + 1, im), h[1], l[1]);
      split2(F(r0, c0 + 8, im), F(r0, c0 + 9, im), h[2], l[2]);
      split2(F(r0 + 8, c0 + 8, im), F(r0 + 8, c0 + 9, im), h[3], l[3]);
      const int base = ((mt * p.KZ + ks) * 4 + 2 * im) * 32 + ln;
      fzf[base] = make_uint4(h[0], h[1], h[2], h[3]);
      fzf[base + 32] = make_uint4(l[0], l[1], l[2], l[3]);
    }
  }
  // t basis in A-fragment order: parts (hi, lo); rows ri * 8 + jt, k slots
  // 2 t4 + {0,1} <-> t = 16 ks + 4 t4 + {0,1} and 2 t4 + 8 + {0,1} <-> + {2,3}
  uint4* ftf = reinterpret_cast<uint4*>(sm + p.o_ft);  // [KT][2 parts][32 lanes]
  for (int e = tid; KTR == 0 && e < p.KT * 32; e += kTzThreads) {
    const int ln = e & 31, ks = e >> 5;
    const int jt = ln >> 2, t0 = 16 * ks + 4 * (ln & 3);
    auto F = [&](int ri, int t) -> float {
      if (jt >= p.Jt || t >= p.Nt) return 0.f;
      const float2 f = p.Ft[(long long)jt * p.Nt + t];
      return rnd<TF>(ri ? f.y : f.x);
    };
    uint32_t h[4], l[4];
    split2(F(0, t0), F(0, t0 + 1), h[0], l[0]);
    split2(F(1, t0), F(1, t0 + 1), h[1], l[1]);
    split2(F(0, t0 + 2), F(0, t0 + 3), h[2], l[2]);
    split2(F(1, t0 + 2), F(1, t0 + 3), h[3], l[3]);
    ftf[(2 * ks) * 32 + ln] = make_uint4(h[0], h[1], h[2], h[3]);
    ftf[(2 * ks + 1) * 32 + ln] = make_uint4(l[0], l[1], l[2], l[3]);
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      tma::mbar_init(&full[s], 1);
      tma::mbar_init(&empty[s], 1);
    }
    *abort_flag = 0;
    *issued = 0;
    tma::fence_mbar_init();
  }
  __syncthreads();

  const long long nmine = (p.nunits > blockIdx.x)
                              ? (p.nunits - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      long long g = 0;
      const long long nstages = nmine * p.NCH;
      for (; g < nstages; ++g) {
        const int s = (int)(g % S);
        if (g >= S && !tma::mbar_wait(&empty[s], (uint32_t)(((g - S) / S) & 1), kTzWait)) {
          atomicExch(p.err, 1);
          *abort_flag = 1;
          break;
        }
        if (*abort_flag) break;
        const long long u = blockIdx.x + (long long)((int)g / p.NCH) * gridDim.x;
        const int ch = (int)g % p.NCH;
        const long long c0 = u * p.G;
        const long long nc = min((long long)p.G, p.ncol - c0);
        const int rows = min(p.zc, p.Nz - ch * p.zc);  // the last chunk may be shorter
        const uint32_t bytes = (p.NCH > 1) ? (uint32_t)(rows * p.Nt * 4)
                                           : (uint32_t)(nc * p.col_floats * 4);
        const float* src = p.in + c0 * p.col_floats + (long long)ch * p.zc * p.Nt;
        tma::mbar_arrive_expect_tx(&full[s], bytes);
        tma::bulk_g2s(sm + p.o_ring + (size_t)s * p.stage_bytes, src, bytes, &full[s]);
        __threadfence_block();
        *issued = (int)g + 1;
      }
      // every copy this CTA started has landed before its shared memory is released
      for (long long q = (g > S ? g - S : 0); q < g; ++q)
        (void)tma::mbar_wait(&full[q % S], (uint32_t)((q / S) & 1), kTzWait);
    }
    return;
  }

  // ---------------- consumers ----------------
  const int cw = warp - 1;
  const int Nt = p.Nt, Nz = p.Nz;
  // register copy of the t basis fragments (KTR > 0), same layout as the table
  uint4 frh[KTR > 0 ? KTR : 1], frl[KTR > 0 ? KTR : 1];
#pragma unroll
  for (int ks = 0; ks < (KTR > 0 ? KTR : 1); ++ks) {
    const int t0 = 16 * ks + 4 * t4;
    auto F = [&](int ri, int t) -> float {
      if (KTR == 0 || g8 >= p.Jt || t >= Nt || ks >= p.KT) return 0.f;
      const float2 f = p.Ft[(long long)g8 * Nt + t];
      return rnd<TF>(ri ? f.y : f.x);
    };
    uint32_t h[4], l[4];
    split2(F(0, t0), F(0, t0 + 1), h[0], l[0]);
    split2(F(1, t0), F(1, t0 + 1), h[1], l[1]);
    split2(F(0, t0 + 2), F(0, t0 + 3), h[2], l[2]);
    split2(F(1, t0 + 2), F(1, t0 + 3), h[3], l[3]);
    frh[ks] = make_uint4(h[0], h[1], h[2], h[3]);
    frl[ks] = make_uint4(l[0], l[1], l[2], l[3]);
  }
  const bool t_vec4 = (Nt & 3) == 0;  // 16-byte rows; otherwise 8-byte (Nt even)
  const int kzc = p.zc / 16;  // z k-steps per staged chunk
  bool ok = true;
  for (int cu = cw; cu < (int)nmine && ok; cu += kTzWarps) {
    const long long u = blockIdx.x + (long long)cu * gridDim.x;
    const long long c0 = u * p.G;
    const int nc = (int)min((long long)p.G, p.ncol - c0);
    for (int cl = 0; cl < nc && ok; ++cl) {
      float tre[MZ][4], tim[MZ][4];
#pragma unroll
      for (int mt = 0; mt < MZ; ++mt)
#pragma unroll
        for (int q = 0; q < 4; ++q) tre[mt][q] = tim[mt][q] = 0.f;
      for (int ch = 0; ch < p.NCH; ++ch) {
        // the stage of this chunk (a whole unit of G columns when NCH = 1)
        const int g = cu * p.NCH + ch;
        const int s = g % S;
        if ((p.NCH > 1 || cl == 0) &&
            (!tz_wait_issued(issued, abort_flag, g) ||
             !tma::mbar_wait(&full[s], (uint32_t)((g / S) & 1), kTzWait) || *abort_flag)) {
          if (lane == 0) {
            atomicExch(p.err, 1);
            *abort_flag = 1;
          }
          ok = false;
          break;
        }
        const float* xs = reinterpret_cast<const float*>(sm + p.o_ring + (size_t)s * p.stage_bytes) +
                          (size_t)cl * p.col_floats;
        const int kz_end = min(ch * kzc + kzc, p.KZ);
        for (int kl = 0; ch * kzc + kl < kz_end; ++kl) {
          const int kz = ch * kzc + kl;
          // t stage of z = 16 kz .. 16 kz + 15 (two n-tiles; staged rows 16 kl ..);
          // rows past Nz and times past Nt enter as zeros
          float pc[2][4];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int q = 0; q < 4; ++q) pc[h][q] = 0.f;
            const bool zin = 16 * kz + 8 * h + g8 < Nz;
            const float* row = xs + (size_t)(16 * kl + 8 * h + g8) * Nt;
#pragma unroll
            for (int ks = 0; ks < (KTR > 0 ? KTR : kTzKTMax); ++ks) {
              if (ks >= p.KT) break;
              const int tt = 16 * ks + 4 * t4;
              float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
              if (zin && tt < Nt) {
                if (t_vec4) {
                  v = *reinterpret_cast<const float4*>(row + tt);
                } else {
                  const float2 a = *reinterpret_cast<const float2*>(row + tt);
                  v.x = a.x;
                  v.y = a.y;
                  if (tt + 2 < Nt) {
                    const float2 b2 = *reinterpret_cast<const float2*>(row + tt + 2);
                    v.z = b2.x;
                    v.w = b2.y;
                  }
                }
              }
              const uint4 fh = KTR > 0 ? frh[KTR > 0 ? ks : 0] : ftf[(2 * ks) * 32 + lane];
              uint32_t bh0, bl0, bh1, bl1;
              split2(rnd<TF>(v.x), rnd<TF>(v.y), bh0, bl0);
              split2(rnd<TF>(v.z), rnd<TF>(v.w), bh1, bl1);
              if (SPLIT) {
                const uint4 fl = KTR > 0 ? frl[KTR > 0 ? ks : 0] : ftf[(2 * ks + 1) * 32 + lane];
                mma16(pc[h], fl.x, fl.y, fl.z, fl.w, bh0, bh1);
                mma16(pc[h], fh.x, fh.y, fh.z, fh.w, bl0, bl1);
              }
              mma16(pc[h], fh.x, fh.y, fh.z, fh.w, bh0, bh1);
            }
          }
          // z stage k-step kz: B fragments straight from the t-stage accumulators
          uint32_t rh0, rl0, rh1, rl1, ih0, il0, ih1, il1;
          split2(rnd<TF>(pc[0][0]), rnd<TF>(pc[0][1]), rh0, rl0);  // P_re, z + 0..7
          split2(rnd<TF>(pc[1][0]), rnd<TF>(pc[1][1]), rh1, rl1);  // P_re, z + 8..15
          split2(rnd<TF>(pc[0][2]), rnd<TF>(pc[0][3]), ih0, il0);  // P_im
          split2(rnd<TF>(pc[1][2]), rnd<TF>(pc[1][3]), ih1, il1);
          const uint32_t nh0 = ih0 ^ 0x80008000u, nh1 = ih1 ^ 0x80008000u;  // -P_im
          const uint32_t nl0 = il0 ^ 0x80008000u, nl1 = il1 ^ 0x80008000u;
#pragma unroll
          for (int mt = 0; mt < MZ; ++mt) {
            const int base = ((mt * p.KZ + kz) * 4) * 32 + lane;
            const uint4 arh = fzf[base], arl = fzf[base + 32];
            const uint4 aih = fzf[base + 64], ail = fzf[base + 96];
            float dr[4] = {0.f, 0.f, 0.f, 0.f}, di[4] = {0.f, 0.f, 0.f, 0.f};
            if (SPLIT) {
              mma16(dr, arl.x, arl.y, arl.z, arl.w, rh0, rh1);
              mma16(dr, arh.x, arh.y, arh.z, arh.w, rl0, rl1);
              mma16(dr, ail.x, ail.y, ail.z, ail.w, nh0, nh1);
              mma16(dr, aih.x, aih.y, aih.z, aih.w, nl0, nl1);
              mma16(di, arl.x, arl.y, arl.z, arl.w, ih0, ih1);
              mma16(di, arh.x, arh.y, arh.z, arh.w, il0, il1);
              mma16(di, ail.x, ail.y, ail.z, ail.w, rh0, rh1);
              mma16(di, aih.x, aih.y, aih.z, aih.w, rl0, rl1);
            }
            mma16(dr, arh.x, arh.y, arh.z, arh.w, rh0, rh1);
            mma16(dr, aih.x, aih.y, aih.z, aih.w, nh0, nh1);
            mma16(di, arh.x, arh.y, arh.z, arh.w, ih0, ih1);
            mma16(di, aih.x, aih.y, aih.z, aih.w, rh0, rh1);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              tre[mt][q] += dr[q];
              tim[mt][q] += di[q];
            }
          }
        }
        if (p.NCH > 1) {  // the chunk has been read
          __syncwarp();
          if (lane == 0) tma::mbar_arrive(&empty[s]);
        }
      }
      if (!ok) break;
      // T[col][kz][jt]: rows kz = 16 mt + g8 (+8), cols jt = 2 t4 + {0, 1}
      float2* oc = p.out + (c0 + cl) * (long long)(p.Jz * p.Jt);
#pragma unroll
      for (int mt = 0; mt < MZ; ++mt)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int kz = 16 * mt + g8 + 8 * hh;
          if (kz >= p.Jz) continue;
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int jt = 2 * t4 + e;
            if (jt < p.Jt) oc[kz * p.Jt + jt] = make_float2(tre[mt][2 * hh + e], tim[mt][2 * hh + e]);
          }
        }
    }
    if (ok && p.NCH == 1) {  // every column of the stage has been read
      __syncwarp();
      if (lane == 0) tma::mbar_arrive(&empty[cu % S]);
    }
  }
}

}  // namespace

// plan: stage columns G (a stage holds at least 8 KB), ring depth S, offsets
// plan: stages of about 16 KB (G whole columns, or a column in NCH chunks of
// zc = 16 kzc rows, the last chunk shorter), ring depth S, table offsets
static bool tz_mma_plan(const Dims& d, TzM& k, size_t& smem) {
  k.Nz = (int)d.Nz;
  k.Nt = (int)d.Nt;
  k.Jz = (int)d.Jz;
  k.Jt = (int)d.Jt;
  k.KT = (int)((d.Nt + 15) / 16);
  k.KZ = (int)((d.Nz + 15) / 16);
  const int MZ = (int)((d.Jz + 15) / 16);
  k.col_floats = (uint32_t)(d.Nz * d.Nt);
  const size_t colb = 4 * (size_t)k.col_floats;
  const size_t target = 16 * 1024;  // stage bytes (fewer, larger bulk copies measured faster)
  if (colb > target) {
    const int nch = (int)((colb + target - 1) / target);
    const int kzc = (k.KZ + nch - 1) / nch;
    k.NCH = (k.KZ + kzc - 1) / kzc;
    k.zc = 16 * kzc;
    k.G = 1;
    k.stage_bytes = (uint32_t)(4 * (size_t)std::min<int64_t>(k.zc, d.Nz) * d.Nt);
  } else {
    k.NCH = 1;
    k.zc = (int)(16 * k.KZ);
    k.G = (int)std::max<size_t>(1, target / colb);
    k.stage_bytes = (uint32_t)(k.G * colb);
  }
  const size_t fzb = (size_t)(MZ <= 1 ? 1 : MZ <= 2 ? 2 : 4) * k.KZ * 4 * 32 * 16;
  const size_t ftb = k.KT > 4 ? (size_t)k.KT * 2 * 32 * 16 : 0;  // registers up to 4 k-steps
  k.o_fz = 0;
  k.o_ft = (uint32_t)((fzb + 127) / 128 * 128);
  k.o_ring = (uint32_t)((k.o_ft + ftb + 127) / 128 * 128);
  const size_t budget = 227 * 1024 / tz_ctas(MZ) - k.o_ring - 1024;
  k.S = (int)std::min<size_t>(32, budget / k.stage_bytes);
  if (k.S < 2) return false;
  k.o_bar = (uint32_t)(k.o_ring + (size_t)k.S * k.stage_bytes);
  smem = k.o_bar + 16 * (size_t)k.S + 16;
  return smem <= 227 * 1024;
}

bool fwd_tz_mma_supported(const Dims& d, char* why, size_t nwhy) {
  const char* r = nullptr;
  if (d.Nt % 2 != 0 || d.Nt > 16 * kTzKTMax)
    r = "the tensor-core t stage needs Nt even and at most 128";
  else if ((d.Nz * d.Nt) % 4 != 0)
    r = "the tensor-core t stage needs Nz * Nt a multiple of 4 (16-byte column copies)";
  else if (d.Jt > 8)
    r = "the tensor-core t stage needs mt <= 8";
  else if (d.Jz > 64)
    r = "the tensor-core z stage needs 2 mz <= 64";
  if (!r) {
    TzM k{};
    size_t smem = 0;
    if (!tz_mma_plan(d, k, smem)) r = "a column of Nz x Nt floats does not fit the staging ring";
  }
  if (r && why) snprintf(why, nwhy, "%s", r);
  return r == nullptr;
}

template <int MZ, int KTR, bool SPLIT, bool TF>
static cudaError_t launch_tz_t(const TzM& k, size_t smem, const char* name, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_fwd_tz_mma<MZ, KTR, SPLIT, TF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid =
      (int)std::max<long long>(1, std::min<long long>((long long)tz_ctas(MZ) * sm_count(), k.nunits));
  FNO_LAUNCH(name, (k_fwd_tz_mma<MZ, KTR, SPLIT, TF>), grid, kTzThreads, smem, s, k);
  return cudaSuccess;
}

template <int MZ, int KTR>
static cudaError_t launch_tz_k(const TzM& k, size_t smem, bool split, bool tf32, cudaStream_t s) {
  if (tf32) return launch_tz_t<MZ, KTR, true, true>(k, smem, "fno_fwd_tz_mma_tf32", s);
  if (split) return launch_tz_t<MZ, KTR, true, false>(k, smem, "fno_fwd_tz_mma_bf16x3", s);
  return launch_tz_t<MZ, KTR, false, false>(k, smem, "fno_fwd_tz_mma_bf16", s);
}

template <int MZ>
static cudaError_t launch_tz_m(const TzM& k, size_t smem, bool split, bool tf32, cudaStream_t s) {
  if (k.KT <= 2) return launch_tz_k<MZ, 2>(k, smem, split, tf32, s);
  if (k.KT <= 4) return launch_tz_k<MZ, 4>(k, smem, split, tf32, s);
  return launch_tz_k<MZ, 0>(k, smem, split, tf32, s);
}

cudaError_t launch_fwd_tz_mma(const float* in, float2* out, int64_t ncol, const Dims& d,
                              const float2* ft, const float2* fz, bool split, bool tf32, int* err,
                              cudaStream_t s) {
  if (ncol <= 0) return cudaSuccess;
  TzM k{};
  size_t smem = 0;
  if (!tz_mma_plan(d, k, smem)) return cudaErrorInvalidValue;
  k.in = in;
  k.out = out;
  k.Ft = ft;
  k.Fz = fz;
  k.err = err;
  k.ncol = ncol;
  k.nunits = (ncol + k.G - 1) / k.G;
  const int MZ = (int)((d.Jz + 15) / 16);
  if (MZ <= 1) return launch_tz_m<1>(k, smem, split, tf32, s);
  if (MZ <= 2) return launch_tz_m<2>(k, smem, split, tf32, s);
  return launch_tz_m<4>(k, smem, split, tf32, s);
}

}  // namespace fno
