// fno_tc.cu -- the last stage of the inverse transform of Alg. 2 (inverse z,
// then inverse t; Sec. IV-C runs the inverse as the adjoint of the forward
// DFT) fused with the block's pointwise 1x1 channel linear, bias and GELU, on
// the 5th-generation tensor cores: tcgen05.mma with FP32 accumulators in
// tensor memory (TMEM), operands staged in shared memory by the TMA engine
// and by converter warps.
//
// Work unit: a tile of 128 consecutive points of one (b, x, y) column (128/Nt
// whole z-planes; TMEM lane = point), and a group of 4 tiles (16 planes at
// Nt = 32).  Per group and tile:
//   stage 1 (inverse z, once per group):
//     QT[(o, jt)][(plane, re/im)] = sum_(jz, re/im) U'[(o, jt)][(jz, re/im)] Bz[(plane, re/im)][(jz, re/im)]
//     A = the column's spectrum U1 (rebuilt when the column changes), B = the
//     z basis of the group's planes (a global table, TMA bulk copy).
//   stage 2 (inverse t, once per group, the group's 4 tiles side by side in N):
//     D2[p][(tile, o)] = sum_plane sum_k2 T_plane[p][k2] Q[tile, plane][o][k2]
//     T_plane: the t basis (c(kt)/N cos, -c(kt)/N sin) on the rows of one
//     plane of the tile and zero elsewhere -- one zero-padded buffer read
//     through descriptor windows shifted by whole planes.
//   1x1 (per tile): D1[p][o] = sum_i X[i][p] W_lin[i][o]   (kind::tf32)
//   epilogue (per tile): A = D1 + D2 + bias; FWD z = GELU(A) (and GELU'(A) in
//     a training forward); DX, SPECTRAL: the sum itself.  A thread owns one
//     point, so each warp store is 128 consecutive bytes of one channel.
//
// Warp roles (16 warps): 0 TMA producer (x tiles, basis slices, spectra);
// 1 and 3 issue the 1x1 MMAs of the even and the odd tiles (1 also owns the
// TMEM allocation); 2 issues the stage-1 and stage-2 MMAs; 4-7 build operands
// (x tile -> TF32 big and small parts in TMEM, spectrum -> U', QT (TMEM) ->
// stage-2 operand in shared memory); 8-15 the epilogue.  The roles hand work over
// through mbarriers only.  A thread waits about 60-170 SM cycles between two
// tcgen05.mma it issues (measured), while the SM accepts one every ~40
// cycles at N <= 64, so three threads issue and every descriptor is formed
// once, outside the loops, and advanced by additions.
//
// Precision.  Split BF16: stages 1 and 2 as hi + lo with three products
// (hi.hi + hi.lo + lo.hi); the 1x1 as 3xTF32 (x = big + small, W likewise,
// big.big + big.small + small.big), FP32-like.  TF32: operands rounded to
// TF32, then stages 1 and 2 as split BF16 (exact for TF32 values up to the
// lo.lo term) and one TF32 product in the 1x1.  (The kernel also has a one-
// product BF16 form; the library runs plain BF16 on the mma.sync epilogue,
// which measured faster for it.)
//
// Every wait is bounded (about 2 s of SM clocks) and watches a CTA abort flag:
// a role that gives up raises it and the error word, every role then leaves
// its loop, the MMA issuers wait for their own MMAs and the producer for its
// copies, and the TMEM allocation is released before the kernel returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdio>

#include "fno_internal.h"
#include "tma.h"
#include "umma.h"
#include "warp_mma.h"

namespace fno {

cudaError_t encode_x_map(CUtensorMap* map, const float* base, long long chan, long long rows,
                         int box_rows);

namespace {

constexpr int kTP = 128;         // points per tile = TMEM lanes
constexpr int kGT = 4;           // tiles per group
constexpr int kWProd = 0, kWIssA = 1, kWIssB = 2, kWIssA2 = 3, kWConv = 4;
// four converter warps, one per TMEM lane quarter (two per quarter measured
// slower: the extra warps took issue slots from the epilogue)
constexpr int kConvWarps = 4;
constexpr int kTcThreads = 32 * (kWConv + kConvWarps + 8);
constexpr long long kTcWait = 4000000000LL;  // about 2 s of SM clocks per wait

// TF32 rounding (nearest, ties away from zero; see warp_mma.h)
__device__ __forceinline__ float tf32_rna(float x) { return wm::tf32_round(x); }
template <bool TF>
__device__ __forceinline__ float rnd_tf(float x) {
  return TF ? tf32_rna(x) : x;
}
// hi/lo BF16 split of two floats packed in pairs (first value in the low half)
__device__ __forceinline__ void split2_bf16(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

}  // namespace

struct EpiTc {
  CUtensorMap tmx;       // the 1x1 input as rows [B * Cl][chan], boxes of Cl rows x 128 points
  EpiArgs a;
  int* err;
  const uint16_t* bz;    // z basis images per plane group: [ngz][hi, lo][NS1 x KZ1] (operand layout)
  long long NxNy, plane, chan, ngroups, gpc;
  int Nz, Nt, Jz, Jt, JZT, ZB, zb_shift, GP, Cs, Cl, nMB, KZ1, NS1, N1, N2, KL, S, Ch;
  uint32_t sbo_u, sbo_a1, sbo_b1;
  uint32_t o_x, x_bytes;    // x ring: S stages of Cl x 128 FP32
  uint32_t o_u1, u1_bytes;  // staged spectrum of one column [Cs][Jz][Jt] complex
  uint32_t o_bz, bz_part;   // z basis: [slot 2][hi, lo]
  uint32_t o_a1;            // start of the zero-initialised operand buffers
  uint32_t o_b1, b1_part;   // W_lin operand: [big, small] N1 x KL TF32
  uint32_t o_us, us_part;   // spectrum operand U': [hi, lo] (nMB 128) x KZ1 BF16
  uint32_t o_tb, tb_part;   // t basis band: [hi, lo] (256 - Nt) x 16 BF16
  uint32_t o_b2, b2_part;   // stage-2 operand: [hi, lo][plane ZB] N2 x 16 BF16
  uint32_t o_bias, o_bar, smem;
  uint32_t t_d1, t_d2, t_qt, t_a1, a1_cols, tcols;
};

// One bounded wait by the calling thread, also ending when the CTA aborts.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (tma::mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 8; ++i)
      if (tma::mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kTcWait) return false;
  }
}
// The same for a whole warp: the decision is uniform over the warp.
__device__ __forceinline__ bool tc_wait_warp(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  const bool ok = tc_wait(bar, parity, abort_flag);
  return __all_sync(0xffffffffu, ok);
}

// CH: channel slots per epilogue thread (a compile-time count, so that the
// per-value chains of the epilogue interleave; the stores are predicated)
template <int MODE, bool SPLIT, bool X3, bool TF, int CH>
__global__ void __launch_bounds__(kTcThreads, 1) k_epi_tc(const __grid_constant__ EpiTc k) {
  constexpr bool LIN = MODE != EPI_SPECTRAL;
  constexpr int NCV = kConvWarps, kWEpi = kWConv + NCV;
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const EpiArgs& a = k.a;
  const int S = k.S;
  uint64_t* xfull = reinterpret_cast<uint64_t*>(sm + k.o_bar);
  uint64_t* xempty = xfull + S;
  uint64_t* u1full = xempty + S;
  uint64_t* u1empty = u1full + 1;
  uint64_t* bzfull = u1empty + 1;  // [2]
  uint64_t* bzempty = bzfull + 2;  // [2]
  uint64_t* a1full = bzempty + 2;  // [2]
  uint64_t* a1empty = a1full + 2;  // [2]
  uint64_t* s1go = a1empty + 2;
  uint64_t* qtfull = s1go + 1;
  uint64_t* b2full = qtfull + 1;
  uint64_t* b2empty = b2full + 1;
  uint64_t* d1full = b2empty + 1;   // [2]
  uint64_t* d1empty = d1full + 2;   // [2]
  uint64_t* d2full = d1empty + 2;   // [2]
  uint64_t* d2empty = d2full + 2;   // [2]
  uint64_t* fin = d2empty + 2;      // [3]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 3);
  volatile int* s_abort = reinterpret_cast<volatile int*>(tslot + 1);
  float* sbias = reinterpret_cast<float*>(sm + k.o_bias);

  // TMA destinations and MMA operands need the window 128-byte aligned:
  // refuse (uniformly, before anything is issued) rather than fault
  if ((tma::smem_u32(sm) & 127u) != 0u) {
    if (tid == 0 && k.err) atomicExch(k.err, 2);
    return;
  }
  const uint32_t s_base = tma::smem_u32(sm);
  auto raise = [&]() {
    *s_abort = 1;
    if (k.err) atomicExch(k.err, 1);
  };

  // ---- set-up: barriers, TMEM, constant operands --------------------------
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      tma::mbar_init(&xfull[i], 1);
      tma::mbar_init(&xempty[i], NCV);
    }
    tma::mbar_init(u1full, 1);
    tma::mbar_init(u1empty, NCV);
    for (int i = 0; i < 2; ++i) {
      tma::mbar_init(&bzfull[i], 1);
      tma::mbar_init(&bzempty[i], 1);
      tma::mbar_init(&a1full[i], NCV);
      tma::mbar_init(&a1empty[i], 1);
      tma::mbar_init(&d1full[i], 1);
      tma::mbar_init(&d1empty[i], 8);
      tma::mbar_init(&d2full[i], 1);
      tma::mbar_init(&d2empty[i], 8);
    }
    for (int i = 0; i < 3; ++i) tma::mbar_init(&fin[i], 1);
    tma::mbar_init(s1go, NCV);
    tma::mbar_init(qtfull, 1);
    tma::mbar_init(b2full, NCV);
    tma::mbar_init(b2empty, 1);
    *s_abort = 0;
    tma::fence_mbar_init();
  }
  if (warp == kWIssA) {
    umma::tmem_alloc(tslot, k.tcols);
    umma::tmem_relinquish();
  }
  {
    // operand buffers start at zero: padding rows and columns are never written
    uint4* z4 = reinterpret_cast<uint4*>(sm + k.o_a1);
    const uint32_t n16 = (k.o_bias - k.o_a1) / 16;
    for (uint32_t e = tid; e < n16; e += kTcThreads) z4[e] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();
  if (LIN) {
    // W_lin as the 1x1's B operand: row o, K = input channel i; TF32 big (and small)
    float* b1 = reinterpret_cast<float*>(sm + k.o_b1);
    for (int e = tid; e < k.N1 * k.KL; e += kTcThreads) {
      const int o = e / k.KL, i = e - o * k.KL;
      const float w = (i < k.Cl && o < k.Cs) ? a.wlin[(size_t)i * a.w_si + (size_t)o * a.w_sc] : 0.f;
      const float big = tf32_rna(w);
      const uint32_t off = umma::koff_tf32((uint32_t)o, (uint32_t)i, k.sbo_b1) / 4u;
      b1[off] = big;
      if (X3) b1[k.b1_part / 4u + off] = w - big;
    }
  }
  {
    // t basis band: row r holds T[t = r - (128 - Nt)][k2] (zero outside the plane),
    // k2 = 2 jt + (0: c/N cos, 1: -c/N sin)
    uint16_t* tb = reinterpret_cast<uint16_t*>(sm + k.o_tb);
    const int r0 = kTP - k.Nt;
    for (int e = tid; e < k.Nt * 16; e += kTcThreads) {
      const int t = e >> 4, kk = e & 15, jt = kk >> 1;
      float v = 0.f;
      if (jt < k.Jt) {
        const float2 f = a.It[(size_t)jt * k.Nt + t];
        v = rnd_tf<TF>((kk & 1) ? -f.y : f.x);
      }
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
      const uint32_t off = umma::koff_bf16((uint32_t)(r0 + t), (uint32_t)kk, 256u) / 2u;
      tb[off] = *reinterpret_cast<const uint16_t*>(&h);
      tb[k.tb_part / 2u + off] = *reinterpret_cast<const uint16_t*>(&l);
    }
  }
  for (int o = tid; o < 32; o += kTcThreads) sbias[o] = (MODE == EPI_FWD && o < k.Cs) ? a.bias[o] : 0.f;
  tma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tbase = *tslot;

  const long long g_begin = k.ngroups * blockIdx.x / gridDim.x;
  const long long g_end = k.ngroups * (blockIdx.x + 1) / gridDim.x;
  const int G = (int)(g_end - g_begin);
  auto col_of = [&](int gl) -> long long { return (g_begin + gl) / k.gpc; };

  // QT (TMEM, rows (o, jt), columns (plane, re/im)) -> stage-2 operand B2, done
  // by the converter warps (all planes of their TMEM lane quarter; converting in
  // the epilogue warps measured slower).  Per thread, constant over the kernel:
  // its row (o, jt) in each M-block and the B2 word offsets of that row in the
  // four tiles' column blocks.
  const int q = warp & 3;
  bool qv[2];
  uint32_t jrow[2][4];
#pragma unroll
  for (int mb = 0; mb < 2; ++mb) {
    const int m = mb * kTP + 32 * q + lane, o = m >> 3, jt = m & 7;
    qv[mb] = (mb < k.nMB) && (o < k.Cs);
#pragma unroll
    for (int j = 0; j < kGT; ++j)
      jrow[mb][j] = qv[mb] ? umma::koff_bf16((uint32_t)(j * k.Cs + o), (uint32_t)(2 * jt), 256u) / 4u : 0u;
  }
  const uint32_t zstride = (uint32_t)k.N2 * 8u, lo_words = k.b2_part / 4u;
  auto conv_qt = [&](int gl) -> bool {
    if (!tc_wait_warp(qtfull, (uint32_t)(gl & 1), s_abort)) return false;
    if (gl >= 1 && !tc_wait_warp(b2empty, (uint32_t)((gl - 1) & 1), s_abort)) return false;
    umma::fence_after_sync();
    uint32_t* b2 = reinterpret_cast<uint32_t*>(sm + k.o_b2);
    // one (re, im) pair of plane pl = j ZB + zz: hi and lo BF16 pairs into B2
    auto put = [&](int mb, int j, int zz, uint32_t re, uint32_t im) {
      uint32_t h, l;
      split2_bf16(rnd_tf<TF>(__uint_as_float(re)), rnd_tf<TF>(__uint_as_float(im)), h, l);
      const uint32_t off = jrow[mb][j] + (uint32_t)zz * zstride;
      b2[off] = h;
      b2[lo_words + off] = l;
    };
#pragma unroll
    for (int mb = 0; mb < 2; ++mb) {
      if (mb >= k.nMB || mb * kTP + 32 * q >= k.Cs * 8) continue;  // uniform over the warp
      const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + k.t_qt + (uint32_t)(mb * k.NS1);
      if (k.ZB == 4) {
        // 16 planes (4 tiles x 4 planes): 32 columns in two halves
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          uint32_t v[16];
          umma::tmem_ld16(ta + (uint32_t)(16 * hf), v);
          umma::tmem_ld_wait();
          if (qv[mb]) {
#pragma unroll
            for (int pp = 0; pp < 8; ++pp) {
              const int pl = 8 * hf + pp;
              put(mb, pl >> 2, pl & 3, v[2 * pp], v[2 * pp + 1]);
            }
          }
        }
      } else {
        // 32 planes (4 tiles x 8 planes): 64 columns in two halves
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          uint32_t v[32];
          umma::tmem_ld16(ta + (uint32_t)(32 * hf), *reinterpret_cast<uint32_t(*)[16]>(&v[0]));
          umma::tmem_ld16(ta + (uint32_t)(32 * hf + 16), *reinterpret_cast<uint32_t(*)[16]>(&v[16]));
          umma::tmem_ld_wait();
          if (qv[mb]) {
#pragma unroll
            for (int pp = 0; pp < 16; ++pp) {
              const int pl = 16 * hf + pp;
              put(mb, pl >> 3, pl & 7, v[2 * pp], v[2 * pp + 1]);
            }
          }
        }
      }
    }
    umma::fence_before_sync();
    tma::fence_proxy_async();
    __syncwarp();
    if (lane == 0) tma::mbar_arrive(b2full);
    return true;
  };

  if (warp == kWProd) {
    // ======================= producer: TMA copies ===========================
    if (lane == 0 && G > 0) {
      bool ok = true;
      int u1_uses = 0;
      int bz_uses[2] = {0, 0};
      int x_uses_total = 0;
      unsigned char* u1s = sm + k.o_u1;
      const uint32_t jzt_bytes = (uint32_t)k.JZT * 8u;
      auto issue_u1 = [&](long long col) -> bool {
        if (u1_uses > 0 && !tc_wait(u1empty, (uint32_t)((u1_uses - 1) & 1), s_abort)) return false;
        const long long b = col / k.NxNy, xy = col - b * k.NxNy;
        tma::fence_proxy_async();
        tma::mbar_arrive_expect_tx(u1full, jzt_bytes * (uint32_t)k.Cs);
        for (int o = 0; o < k.Cs; ++o)
          tma::bulk_g2s(u1s + (size_t)o * jzt_bytes, a.U + ((b * k.Cs + o) * k.NxNy + xy) * k.JZT, jzt_bytes,
                        u1full);
        ++u1_uses;
        return true;
      };
      auto issue_bz = [&](int gl) -> bool {
        const int slot = gl & 1;
        if (bz_uses[slot] > 0 && !tc_wait(&bzempty[slot], (uint32_t)((bz_uses[slot] - 1) & 1), s_abort))
          return false;
        const long long pg = (g_begin + gl) % k.gpc;
        tma::fence_proxy_async();
        tma::mbar_arrive_expect_tx(&bzfull[slot], 2u * k.bz_part);
        tma::bulk_g2s(sm + k.o_bz + (size_t)slot * 2u * k.bz_part, k.bz + (size_t)pg * (k.bz_part / 2u) * 2u,
                      2u * k.bz_part, &bzfull[slot]);
        ++bz_uses[slot];
        return true;
      };
      // the spectrum and z basis of group gl + 2 are staged during group gl:
      // the converters build stage 1's operand two groups ahead
      long long prev_col = col_of(0);
      ok = issue_u1(prev_col) && issue_bz(0);
      if (ok && G > 1) {
        ok = issue_bz(1);
        if (ok && col_of(1) != prev_col) {
          prev_col = col_of(1);
          ok = issue_u1(prev_col);
        }
      }
      for (int gl = 0; ok && gl < G; ++gl) {
        if (gl + 2 < G) {
          ok = issue_bz(gl + 2);
          const long long c2 = col_of(gl + 2);
          if (ok && c2 != prev_col) {
            ok = issue_u1(c2);
            prev_col = c2;
          }
        }
        if (LIN) {
          const long long gid = g_begin + gl, col = gid / k.gpc, pg = gid - col * k.gpc;
          const long long b = col / k.NxNy, xy = col - b * k.NxNy;
          for (int j = 0; ok && j < kGT; ++j) {
            const int t = kGT * gl + j, s = t % S, n = t / S;
            if (n > 0 && !tc_wait(&xempty[s], (uint32_t)((n - 1) & 1), s_abort)) {
              ok = false;
              break;
            }
            const long long c0 = xy * k.plane + (pg * k.GP + (long long)j * k.ZB) * k.Nt;
            tma::fence_proxy_async();
            tma::mbar_arrive_expect_tx(&xfull[s], k.x_bytes);
            tma::tma_load_2d(sm + k.o_x + (size_t)s * k.x_bytes, &k.tmx, (int)c0, (int)(b * k.Cl), &xfull[s]);
            x_uses_total = t + 1;
          }
        }
      }
      if (!ok) raise();
      // every copy this thread started lands before the kernel returns
      for (int s = 0; s < S; ++s) {
        const int n = (x_uses_total > s) ? (x_uses_total - 1 - s) / S + 1 : 0;
        if (n > 0) (void)tma::mbar_wait(&xfull[s], (uint32_t)((n - 1) & 1));
      }
      if (u1_uses > 0) (void)tma::mbar_wait(u1full, (uint32_t)((u1_uses - 1) & 1));
      for (int q = 0; q < 2; ++q)
        if (bz_uses[q] > 0) (void)tma::mbar_wait(&bzfull[q], (uint32_t)((bz_uses[q] - 1) & 1));
    }
  } else if (warp == kWIssA || warp == kWIssA2) {
    // ============= MMA issuers: the 1x1 of the even / the odd tiles ==========
    const int bsel = (warp == kWIssA) ? 0 : 1;
    if (LIN && lane == 0 && G > 0) {
      const uint32_t id1 = umma::idesc(umma::kFmtTF32, kTP, k.N1);
      // the x operand in TMEM (lane = point, column = channel): [buf][big, small];
      // B descriptors advance by 16-byte units in their address field
      const uint32_t abig = tbase + k.t_a1 + (uint32_t)bsel * k.a1_cols, asmall = abig + (uint32_t)k.KL;
      const uint64_t bbig = umma::sdesc(s_base + k.o_b1, 128u, k.sbo_b1);
      const uint64_t bsmall = bbig + (k.b1_part >> 4);
      const uint32_t d = tbase + k.t_d1 + (uint32_t)(bsel * k.N1);
      const int nks = k.KL / 8;
      bool ok = true;
      for (int t = bsel; ok && t < kGT * G; t += 2) {
        const int n = t >> 1;
        if (!tc_wait(&a1full[bsel], (uint32_t)(n & 1), s_abort) ||
            (t >= 2 && !tc_wait(&d1empty[bsel], (uint32_t)((n - 1) & 1), s_abort))) {
          ok = false;
          break;
        }
        umma::fence_after_sync();
        for (int ks = 0; ks < nks; ++ks) {
          const uint64_t ko = (uint64_t)(ks * 16);
          const uint32_t ka = (uint32_t)(ks * 8);
          umma::mma_tf32_ts(d, abig + ka, bbig + ko, id1, ks > 0 ? 1u : 0u);
          if (X3) {
            umma::mma_tf32_ts(d, abig + ka, bsmall + ko, id1, 1u);
            umma::mma_tf32_ts(d, asmall + ka, bbig + ko, id1, 1u);
          }
        }
        umma::commit(&d1full[bsel]);
        umma::commit(&a1empty[bsel]);
      }
      if (!ok) raise();
      umma::commit(&fin[2 * bsel]);
      (void)tma::mbar_wait(&fin[2 * bsel], 0u);
    }
  } else if (warp == kWIssB) {
    // ======================= MMA issuer: stages 1 and 2 =====================
    if (lane == 0 && G > 0) {
      const uint32_t id_s1 = umma::idesc(umma::kFmtBF16, kTP, k.NS1);
      const uint32_t id_s2 = umma::idesc(umma::kFmtBF16, kTP, k.N2);
      const uint64_t us_hi = umma::sdesc(s_base + k.o_us, 128u, k.sbo_u), us_lo = us_hi + (k.us_part >> 4);
      const uint64_t bz_hi = umma::sdesc(s_base + k.o_bz, 128u, k.sbo_u);
      const uint64_t tb_hi = umma::sdesc(s_base + k.o_tb, 128u, 256u), tb_lo = tb_hi + (k.tb_part >> 4);
      const uint64_t b2_hi = umma::sdesc(s_base + k.o_b2, 128u, 256u), b2_lo = b2_hi + (k.b2_part >> 4);
      const uint64_t mb_step = (uint64_t)(16u * k.sbo_u) >> 4, bz_slot = (uint64_t)(2u * k.bz_part) >> 4,
                     bz_part = (uint64_t)k.bz_part >> 4;
      auto stage1 = [&](int gl) -> bool {
        const int slot = gl & 1;
        if (!tc_wait(s1go, (uint32_t)(gl & 1), s_abort) ||
            !tc_wait(&bzfull[slot], (uint32_t)((gl >> 1) & 1), s_abort))
          return false;
        umma::fence_after_sync();
        const uint64_t bzh = bz_hi + (uint64_t)slot * bz_slot, bzl = bzh + bz_part;
        for (int mb = 0; mb < k.nMB; ++mb) {
          const uint32_t d = tbase + k.t_qt + (uint32_t)(mb * k.NS1);
          const uint64_t ah = us_hi + (uint64_t)mb * mb_step, al = us_lo + (uint64_t)mb * mb_step;
          for (int ks = 0; ks < k.KZ1 / 16; ++ks) {
            const uint64_t ko = (uint64_t)(ks * 16);
            umma::mma_bf16(d, ah + ko, bzh + ko, id_s1, ks > 0 ? 1u : 0u);
            if (SPLIT) {
              umma::mma_bf16(d, ah + ko, bzl + ko, id_s1, 1u);
              umma::mma_bf16(d, al + ko, bzh + ko, id_s1, 1u);
            }
          }
        }
        umma::commit(qtfull);
        umma::commit(&bzempty[slot]);
        return true;
      };
      auto stage2 = [&](int gl) -> bool {
        const int bsel = gl & 1;
        if (!tc_wait(b2full, (uint32_t)(gl & 1), s_abort) ||
            (gl >= 2 && !tc_wait(&d2empty[bsel], (uint32_t)(((gl >> 1) - 1) & 1), s_abort)))
          return false;
        umma::fence_after_sync();
        const uint32_t d = tbase + k.t_d2 + (uint32_t)(bsel * k.N2);
        for (int zz = 0; zz < k.ZB; ++zz) {
          // the t basis window of plane zz starts (128 - Nt - zz Nt) / 8 row groups in
          const uint64_t ao = (uint64_t)((kTP - k.Nt - zz * k.Nt) / 8) * 16u, bo = (uint64_t)(zz * k.N2 * 2);
          umma::mma_bf16(d, tb_hi + ao, b2_hi + bo, id_s2, zz > 0 ? 1u : 0u);
          if (SPLIT) {
            umma::mma_bf16(d, tb_hi + ao, b2_lo + bo, id_s2, 1u);
            umma::mma_bf16(d, tb_lo + ao, b2_hi + bo, id_s2, 1u);
          }
        }
        umma::commit(&d2full[bsel]);
        umma::commit(b2empty);
        return true;
      };
      bool ok = stage1(0);
      for (int gl = 0; ok && gl < G; ++gl) {
        ok = stage2(gl);
        if (ok && gl + 1 < G) ok = stage1(gl + 1);
      }
      if (!ok) raise();
      umma::commit(&fin[1]);
      (void)tma::mbar_wait(&fin[1], 0u);
    }
  } else if (warp < kWEpi) {
    // ======================= operand converters =============================
    const int ct = tid - 32 * kWConv;  // 0 .. 32 NCV - 1
    bool ok = true;
    int u1_use = 0;
    // U'[(o, jt)][(jz, re/im)] from the staged spectrum [o][jz][jt]
    auto build_us = [&]() -> bool {
      if (!tc_wait_warp(u1full, (uint32_t)(u1_use & 1), s_abort)) return false;
      ++u1_use;
      const float2* u1s = reinterpret_cast<const float2*>(sm + k.o_u1);
      uint32_t* us = reinterpret_cast<uint32_t*>(sm + k.o_us);
      // this thread's (jz, jt) items r = ct, ct + 32 NCV, ... (Jz Jt <= 192)
      for (int r = ct; r < k.JZT; r += 32 * NCV) {
        const int jz = r / k.Jt, jt = r - jz * k.Jt;
        uint32_t off = umma::koff_bf16((uint32_t)jt, (uint32_t)(2 * jz), k.sbo_u) / 4u;
        const float2* src = u1s + r;
        for (int o = 0; o < k.Cs; ++o) {
          // row o * 8 + jt: one 8-row group per output channel
          const float2 u = src[(size_t)o * k.JZT];
          uint32_t h, l;
          split2_bf16(rnd_tf<TF>(u.x), rnd_tf<TF>(u.y), h, l);
          us[off] = h;
          us[k.us_part / 4u + off] = l;
          off += k.sbo_u / 4u;
        }
      }
      tma::fence_proxy_async();
      __syncwarp();
      if (lane == 0) tma::mbar_arrive(u1empty);
      return true;
    };
    // x tile (FP32 [Cl][128]) -> the 1x1's A operand in TMEM, buffer t & 1: this
    // thread's point p = 32 q + lane is TMEM lane p; column = channel (TF32 big,
    // then small)
    auto conv_x = [&](int t) -> bool {
      const int s = t % S, n = t / S, bsel = t & 1;
      if (!tc_wait_warp(&xfull[s], (uint32_t)(n & 1), s_abort)) return false;
      if (t >= 2 && !tc_wait_warp(&a1empty[bsel], (uint32_t)(((t >> 1) - 1) & 1), s_abort)) return false;
      umma::fence_after_sync();
      const float* xs = reinterpret_cast<const float*>(sm + k.o_x + (size_t)s * k.x_bytes);
      const int p = 32 * q + lane;
      const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + k.t_a1 + (uint32_t)bsel * k.a1_cols;
#pragma unroll
      for (int c8 = 0; c8 < 4; ++c8) {
        if (8 * c8 < k.KL) {
          uint32_t big[8], small[8];
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            // rows past Cl read the last row and are zeroed by a select (no branch)
            const int i = 8 * c8 + r;
            const float xv = xs[(size_t)min(i, k.Cl - 1) * kTP + p];
            const float v = (i < k.Cl) ? xv : 0.f;
            const float bg = tf32_rna(v);
            big[r] = __float_as_uint(bg);
            small[r] = __float_as_uint(v - bg);
          }
          umma::tmem_st8(ta + (uint32_t)(8 * c8), big);
          if (X3) umma::tmem_st8(ta + (uint32_t)(k.KL + 8 * c8), small);
        }
      }
      umma::tmem_st_wait();
      umma::fence_before_sync();
      __syncwarp();
      if (lane == 0) {
        tma::mbar_arrive(&a1full[bsel]);
        tma::mbar_arrive(&xempty[s]);
      }
      return true;
    };
    // Arrivals carry no phase, so a warp arrives on s1go for phase p only once
    // phase p - 1 has completed; otherwise a warp running ahead would complete
    // phase p - 1 early, before a slower warp had written its part of U'.
    auto go_s1 = [&](int p) -> bool {
      if (p > 0 && !tc_wait_warp(s1go, (uint32_t)((p - 1) & 1), s_abort)) return false;
      __syncwarp();
      if (lane == 0) tma::mbar_arrive(s1go);
      return true;
    };
    // the stage-1 operand U' of group p; a new column's U' is built once S1 of
    // group p - 1 has read the previous one (qtfull phase p - 1)
    auto stage1_operand = [&](int p) -> bool {
      if (p > 0 && col_of(p) == col_of(p - 1)) return go_s1(p);
      if (p > 0 && !tc_wait_warp(qtfull, (uint32_t)((p - 1) & 1), s_abort)) return false;
      if (!build_us()) return false;
      return go_s1(p);
    };
    if (G > 0) {
      ok = stage1_operand(0);
      ok = ok && conv_qt(0);
      if (ok && G > 1) ok = stage1_operand(1);
      // per group gl: its first x tile, the stage-2 operand of gl + 1, the
      // stage-1 operand of gl + 2, its other x tiles
      for (int gl = 0; ok && gl < G; ++gl) {
        if (LIN) ok = conv_x(kGT * gl);
        if (ok && gl + 1 < G) ok = conv_qt(gl + 1);
        if (ok && gl + 2 < G) ok = stage1_operand(gl + 2);
        if (LIN)
          for (int j = 1; ok && j < kGT; ++j) ok = conv_x(kGT * gl + j);
      }
      if (!ok && lane == 0) raise();
    }
  } else {
    // ======================= epilogue =======================================
    const int h = (warp - kWEpi) >> 2;
    const int p = 32 * q + lane;
    const int c_lo = h * k.Ch;
    const int nc = min(k.Ch, k.Cs - c_lo);
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    float bias_r[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) bias_r[c] = sbias[min(c_lo + c, 31)];
    bool ok = true;
    for (int gl = 0; ok && gl < G; ++gl) {
      const int gsel = gl & 1;
      if (!tc_wait_warp(&d2full[gsel], (uint32_t)((gl >> 1) & 1), s_abort)) {
        ok = false;
        break;
      }
      umma::fence_after_sync();
      const long long gid = g_begin + gl, col = gid / k.gpc, pg = gid - col * k.gpc;
      const long long b = col / k.NxNy, xy = col - b * k.NxNy;
      for (int j = 0; j < kGT; ++j) {
        const int t = kGT * gl + j, tsel = t & 1;
        if (LIN) {
          if (!tc_wait_warp(&d1full[tsel], (uint32_t)((t >> 1) & 1), s_abort)) {
            ok = false;
            break;
          }
          umma::fence_after_sync();
        }
        uint32_t v2[16], v1[16];
        {
          const uint32_t c2 = tbase + lane_addr + k.t_d2 + (uint32_t)(gsel * k.N2 + j * k.Cs + c_lo);
          umma::tmem_ld8(c2, *reinterpret_cast<uint32_t(*)[8]>(&v2[0]));
          if (CH > 8) umma::tmem_ld8(c2 + 8u, *reinterpret_cast<uint32_t(*)[8]>(&v2[8]));
          if (LIN) {
            const uint32_t c1 = tbase + lane_addr + k.t_d1 + (uint32_t)(tsel * k.N1 + c_lo);
            umma::tmem_ld8(c1, *reinterpret_cast<uint32_t(*)[8]>(&v1[0]));
            if (CH > 8) umma::tmem_ld8(c1 + 8u, *reinterpret_cast<uint32_t(*)[8]>(&v1[8]));
          }
          umma::tmem_ld_wait();
        }
        umma::fence_before_sync();
        __syncwarp();
        if (lane == 0) {
          if (LIN) tma::mbar_arrive(&d1empty[tsel]);
          if (j == kGT - 1) tma::mbar_arrive(&d2empty[gsel]);
        }
        const long long tile_ofs = xy * k.plane + (pg * k.GP + (long long)j * k.ZB) * k.Nt + p;
        float* ob = a.out + (b * k.Cs + c_lo) * k.chan + tile_ofs;
        float* gb = (MODE == EPI_FWD && a.gp) ? a.gp + (b * k.Cs + c_lo) * k.chan + tile_ofs : nullptr;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          float v = __uint_as_float(v2[c]);
          if (LIN) v += __uint_as_float(v1[c]);
          float gz = 0.f;
          if (MODE == EPI_FWD) {
            v += bias_r[c];
            float phi2, ex;
            phi2_as(v, phi2, ex);
            gz = fmaf(v * ex, 0.39894228040143268f, 0.5f * phi2);
            v = 0.5f * v * phi2;
          }
          if (c < nc) {
            *ob = v;
            if (MODE == EPI_FWD && gb) *gb = gz;
          }
          ob += k.chan;
          if (MODE == EPI_FWD) gb += k.chan;
        }
      }
    }
    if (!ok && lane == 0) raise();
  }

  // ---- tear-down: every role is done; the TMEM allocation is released -----
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (warp == kWIssA) umma::tmem_dealloc(tbase, k.tcols);
}

// z basis images of every plane group, in the stage-1 B-operand layout:
// row n = 2 plane + part, K = 2 jz + (re, im) of the spectrum:
//   part 0: ( Re Iz, -Im Iz)      part 1: (Im Iz, Re Iz)
__global__ void k_epi_tc_bz(const float2* __restrict__ Iz, int Nz, int Jz, int GP, int NS1, int KZ1,
                            int tf32, int ngz, uint16_t* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int per = NS1 * KZ1;
  if (idx >= ngz * per) return;
  const int pg = idx / per, r = idx - pg * per, n = r / KZ1, kk = r - n * KZ1;
  const int z = pg * GP + (n >> 1), part = n & 1, jz = kk >> 1, rp = kk & 1;
  float v = 0.f;
  if (z < Nz && jz < Jz) {
    const float2 f = Iz[(size_t)z * Jz + jz];
    v = (part == 0) ? (rp == 0 ? f.x : -f.y) : (rp == 0 ? f.y : f.x);
    if (tf32) v = tf32_rna(v);
  }
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
  const uint32_t off = umma::koff_bf16((uint32_t)n, (uint32_t)kk, (uint32_t)KZ1 * 16u) / 2u;
  uint16_t* base = out + (size_t)pg * 2 * per;
  base[off] = *reinterpret_cast<const uint16_t*>(&h);
  base[per + off] = *reinterpret_cast<const uint16_t*>(&l);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static uint32_t al128(uint32_t x) { return (x + 127u) / 128u * 128u; }

static bool tc_plan(const Dims& d, int mode, int Cs, int Cl, EpiTc& k, char* why, size_t nwhy) {
  auto no = [&](const char* m) {
    if (why && nwhy) snprintf(why, nwhy, "tcgen05 epilogue: %s", m);
    return false;
  };
  if (mode != EPI_FWD && mode != EPI_DX && mode != EPI_SPECTRAL) return no("mode");
  const bool lin = mode != EPI_SPECTRAL;
  if (d.Nt != 16 && d.Nt != 32) return no("needs Nt of 16 or 32");
  if (d.Jt > 8) return no("needs mt <= 8");
  if (Cs < 1 || Cs > 32) return no("needs 1..32 output channels");
  if (lin && (Cl < 1 || Cl > 32)) return no("needs 1..32 1x1 inputs");
  k.Nz = (int)d.Nz;
  k.Nt = (int)d.Nt;
  k.Jz = (int)d.Jz;
  k.Jt = (int)d.Jt;
  k.JZT = k.Jz * k.Jt;
  k.ZB = kTP / k.Nt;
  k.zb_shift = (k.ZB == 8) ? 3 : 2;
  k.GP = kGT * k.ZB;
  if (k.Nz % k.GP != 0) return no("needs Nz a multiple of 4 * 128 / Nt");
  k.Cs = Cs;
  k.Cl = lin ? Cl : 0;
  k.nMB = (Cs * 8 + kTP - 1) / kTP;
  k.KZ1 = (2 * k.Jz + 15) / 16 * 16;
  if (k.KZ1 > 48) return no("needs 2 mz <= 24");
  k.NS1 = 2 * k.GP;
  k.N1 = lin ? (Cs <= 16 ? 16 : 32) : 0;
  k.N2 = (kGT * Cs + 15) / 16 * 16;
  k.KL = lin ? (Cl + 7) / 8 * 8 : 0;
  k.Ch = (Cs + 1) / 2;
  k.sbo_u = (uint32_t)k.KZ1 * 16u;
  k.sbo_a1 = (uint32_t)k.KL * 32u;
  k.sbo_b1 = (uint32_t)k.KL * 32u;
  // TMEM columns: D1 [2][N1], D2 [2][N2], QT [nMB][NS1]; epilogue loads read up
  // to 16 columns from the start of a range
  k.t_d1 = 0;
  k.t_d2 = (uint32_t)(2 * k.N1);
  k.t_qt = k.t_d2 + (uint32_t)(2 * k.N2);
  k.t_a1 = k.t_qt + (uint32_t)(k.nMB * k.NS1);
  // the x operand of the 1x1: two buffers of KL TF32 columns (big, and small in split BF16)
  k.a1_cols = lin ? (uint32_t)(k.KL * 2) : 0u;
  uint32_t need = k.t_a1 + 2u * k.a1_cols;
  need = std::max(need, k.t_d2 + (uint32_t)(k.N2 + (kGT - 1) * Cs + k.Ch + 16));
  k.tcols = 32;
  while (k.tcols < need) k.tcols <<= 1;
  if (k.tcols > 512) return no("TMEM columns");
  // shared memory
  const uint32_t x_bytes = lin ? (uint32_t)(k.Cl * kTP * 4) : 0u;
  k.x_bytes = x_bytes;
  k.u1_bytes = (uint32_t)(Cs * k.JZT * 8);
  k.bz_part = (uint32_t)(k.NS1 * k.KZ1 * 2);
  k.b1_part = lin ? (uint32_t)(k.N1 * k.KL * 4) : 0u;
  k.us_part = (uint32_t)(k.nMB * kTP * k.KZ1 * 2);
  k.tb_part = (uint32_t)((2 * kTP - k.Nt) * 16 * 2);
  k.b2_part = (uint32_t)(k.ZB * k.N2 * 16 * 2);
  for (int S = 4; S >= 2; --S) {
    uint32_t o = 0;
    k.o_x = o;
    o = al128(o + (uint32_t)S * x_bytes);
    k.o_u1 = o;
    o = al128(o + k.u1_bytes);
    k.o_bz = o;
    o = al128(o + 4u * k.bz_part);
    k.o_a1 = o;  // zero-initialised from here to o_bias
    k.o_b1 = o;
    o = al128(o + 2u * k.b1_part);
    k.o_us = o;
    o = al128(o + 2u * k.us_part);
    k.o_tb = o;
    o = al128(o + 2u * k.tb_part);
    k.o_b2 = o;
    o = al128(o + 2u * k.b2_part);
    k.o_bias = o;
    o += 32 * 4;
    k.o_bar = o;
    o += (uint32_t)(2 * S + 25) * 8u + 16u;
    if (o <= 227u * 1024u) {
      k.S = S;
      k.smem = o;
      break;
    }
    if (S == 2) return no("shared memory");
  }
  // every MMA operand stays inside its region (host-side check of the
  // descriptor arithmetic): a K-major operand of R rows reads up to byte
  // (R/8 - 1) SBO + LBO + 128 from its start
  auto span = [](uint32_t rows, uint32_t sbo) { return (rows / 8u - 1u) * sbo + 256u; };
  if ((uint32_t)(k.nMB - 1) * 16u * k.sbo_u + (uint32_t)(k.KZ1 / 16 - 1) * 256u + span(kTP, k.sbo_u) > k.us_part)
    return no("stage-1 A operand extent");
  if ((uint32_t)(k.KZ1 / 16 - 1) * 256u + span((uint32_t)k.NS1, k.sbo_u) > k.bz_part)
    return no("stage-1 B operand extent");
  if ((uint32_t)((kTP - k.Nt) / 8) * 256u + span(kTP, 256u) > k.tb_part) return no("stage-2 A operand extent");
  if ((uint32_t)(k.ZB - 1) * (uint32_t)k.N2 * 32u + span((uint32_t)k.N2, 256u) > k.b2_part)
    return no("stage-2 B operand extent");
  if (lin) {
    if ((uint32_t)(k.KL / 8 - 1) * 256u + span((uint32_t)k.N1, k.sbo_b1) > k.b1_part)
      return no("1x1 B operand extent");
  }
  if (k.Jz * k.Jt * 8 % 16 != 0) return no("spectrum rows must be 16-byte multiples");
  return true;
}

bool epilogue_tc_supported(const Dims& d, int mode, int Cs, int Cl, char* why, size_t nwhy) {
  EpiTc k{};
  return tc_plan(d, mode, Cs, Cl, k, why, nwhy);
}

size_t epilogue_tc_table_bytes(const Dims& d) {
  const int ZB = (d.Nt == 16 || d.Nt == 32) ? (int)(kTP / d.Nt) : 1;
  const int GP = kGT * ZB;
  const int ngz = (int)((d.Nz + GP - 1) / GP);
  const int KZ1 = (int)((2 * d.Jz + 15) / 16 * 16);
  return (size_t)ngz * 2 * (size_t)(2 * GP) * KZ1 * sizeof(uint16_t);
}

template <int MODE, bool SPLIT, bool X3, bool TF, int CH>
static cudaError_t launch_tc_c(const EpiTc& k, cudaStream_t s, const char* name) {
  const void* kern = (const void*)k_epi_tc<MODE, SPLIT, X3, TF, CH>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
  if (e != cudaSuccess) return e;
  long long g = sm_count();
  if (g > k.ngroups) g = k.ngroups;
  if (g < 1) g = 1;
  FNO_LAUNCH(name, (k_epi_tc<MODE, SPLIT, X3, TF, CH>), (int)g, kTcThreads, k.smem, s, k);
  return cudaSuccess;
}

template <int MODE, bool SPLIT, bool X3, bool TF>
static cudaError_t launch_tc_t(const EpiTc& k, cudaStream_t s, const char* name) {
  if (k.Ch <= 8) return launch_tc_c<MODE, SPLIT, X3, TF, 8>(k, s, name);
  if (k.Ch <= 10) return launch_tc_c<MODE, SPLIT, X3, TF, 10>(k, s, name);
  return launch_tc_c<MODE, SPLIT, X3, TF, 16>(k, s, name);
}

template <int MODE>
static cudaError_t launch_tc_m(const EpiTc& k, bool split, bool tf32, cudaStream_t s) {
  static const char* names[3][4] = {
      {"fno_epi_spectral_tc_bf16", "fno_epi_fwd_tc_bf16", "", "fno_epi_dx_tc_bf16"},
      {"fno_epi_spectral_tc_bf16x3", "fno_epi_fwd_tc_bf16x3", "", "fno_epi_dx_tc_bf16x3"},
      {"fno_epi_spectral_tc_tf32", "fno_epi_fwd_tc_tf32", "", "fno_epi_dx_tc_tf32"}};
  static const char* train_names[3] = {"fno_epi_fwd_train_tc_bf16", "fno_epi_fwd_train_tc_bf16x3",
                                       "fno_epi_fwd_train_tc_tf32"};
  const int pv = tf32 ? 2 : (split ? 1 : 0);
  const char* name = (MODE == EPI_FWD && k.a.gp) ? train_names[pv] : names[pv][MODE];
  if (tf32) return launch_tc_t<MODE, true, false, true>(k, s, name);
  return split ? launch_tc_t<MODE, true, true, false>(k, s, name) : launch_tc_t<MODE, false, false, false>(k, s, name);
}

cudaError_t launch_epilogue_tc(const Dims& d, const EpiArgs& a, bool split, bool tf32, void* table, int* err,
                               cudaStream_t s) {
  EpiTc k{};
  if (!tc_plan(d, a.mode, a.Cs, a.Cl, k, nullptr, 0)) return cudaErrorInvalidValue;
  k.a = a;
  k.err = err;
  k.NxNy = d.Nx * d.Ny;
  k.plane = d.Nz * d.Nt;
  k.chan = k.NxNy * k.plane;
  k.gpc = d.Nz / k.GP;
  k.ngroups = d.B * k.NxNy * k.gpc;
  k.bz = static_cast<const uint16_t*>(table);
  if (a.mode != EPI_SPECTRAL) {
    cudaError_t e = encode_x_map(&k.tmx, a.lin_in, k.chan, d.B * (long long)a.Cl, a.Cl);
    if (e != cudaSuccess) return e;
  }
  {
    const int ngz = (int)k.gpc;
    const int total = ngz * k.NS1 * k.KZ1;
    FNO_LAUNCH("fno_epi_tc_tables", k_epi_tc_bz, (total + 255) / 256, 256, 0, s, a.Iz, k.Nz, k.Jz, k.GP, k.NS1,
               k.KZ1, tf32 ? 1 : 0, ngz, static_cast<uint16_t*>(table));
  }
  switch (a.mode) {
    case EPI_SPECTRAL: return launch_tc_m<EPI_SPECTRAL>(k, split, tf32, s);
    case EPI_FWD: return launch_tc_m<EPI_FWD>(k, split, tf32, s);
    default: return launch_tc_m<EPI_DX>(k, split, tf32, s);
  }
}

}  // namespace fno
