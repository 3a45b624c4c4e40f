// fno_da_tz.cu -- the first pass of a block backward after a training forward
// (the backward of Alg. 2's block, Sec. IV-C), in one kernel:
//   dA = dz * GELU'(A)       from the forward's saved GELU'(A), written out;
//   dW_lin[i][o] += sum_p x[i][p] dA[o][p],  db[o] += sum_p dA[o][p]
//                            as per-CTA partial rows (launch_reduce_partials);
//   T1 = the pruned forward DFT over t, then z, of every dA column (the first
//        half of G = (c/N) DFT(dA)), which a separate pass would read back.
//
// Work unit: one (b, x, y) column of every channel, streamed in chunks of 256
// points (ZC = 256 / Nt whole z-planes).  Each input arrives per chunk as one
// TMA copy of a [C rows][9 blocks][32 points] box with the 128-byte swizzle
// (the 16-byte chunk index within a 128-byte line XOR the line index mod 8):
// the copy walks each channel row along 1152 contiguous bytes, which DRAM
// serves at full rate, and with 9 lines per row the eight rows that a tensor
// core fragment reads at one point fall into eight different XOR classes, so
// those loads are free of bank conflicts.  The ninth block is the next chunk's
// first and is not used (it is read again, usually from L2, with that chunk).
//
// Sixteen warps in two roles, handing each chunk over through mbarriers:
//   warps 8-15 ("DFT warps"), warp 8 + v: dA at the points 32 v .. 32 v + 31
//     for every output channel, in place of dz in the ring and to global
//     memory; then, after a barrier of these warps, the t stage of channels
//     o = v, v + 8, v + 16 on mma.sync m16n8k16, whose accumulators of two
//     8-plane n-tiles form the B fragment of one 16-plane z k-step; the z
//     stage's totals stay in registers over the column's chunks and are
//     written at its end ([col][Jz][Jt] complex, the layout of the separate
//     t, z kernel, with the same products in the same order).
//   warps 0-7 ("dW warps"), warp w, once the chunk's dA is in place: its
//     share of (dW_lin, db), the 32 points of block w, on mma.sync m16n8k8
//     TF32 with split operands (big.big + big.small + small.big, as accurate
//     as FP32 products), per chunk from zero, Kahan-folded.
// Thread 0 starts the copies of the first S chunks; afterwards the warp that
// finishes a chunk last (a count per slot) starts the copy of the chunk S
// places later into its slot.
//
// Every wait is bounded (about 2 s of SM clocks) and watches a CTA abort flag:
// a role that gives up raises it and *err, every role leaves its loop, the
// copies in flight are waited for (bounded), and the kernel returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdio>

#include "fno_internal.h"
#include "tma.h"
#include "warp_mma.h"

namespace fno {

namespace {

constexpr int kDtWarpsA = 8;                  // (dW_lin, db) warps
constexpr int kDtWarpsB = 8;                  // dA and t, z DFT warps
constexpr int kDtThreads = 32 * (kDtWarpsA + kDtWarpsB);
constexpr int kDtPoints = 256;                // points per chunk (8 blocks of 32)
constexpr int kDtBoxBlocks = 9;               // blocks per row of a staged box
constexpr uint32_t kDtRow = 128u * kDtBoxBlocks;  // bytes per staged row
constexpr int kDtCPW = 3;                     // channels per DFT warp (Co <= 24)
constexpr long long kDtWait = 4000000000LL;   // about 2 s of SM clocks

struct DaTz {
  CUtensorMap mx, mdz, mgp;       // [rows][9 blocks][32 points] boxes, 128-byte swizzle
  const float2* Ft;               // [Jt][Nt] t basis of the adjoint DFT (scaled)
  const float2* Fz;               // [Jz][Nz]
  float* da;                      // [B][Co][chan]
  float2* out;                    // [B Co Nx Ny][Jz][Jt]
  float* part;                    // [grid][Ci Co + Co]
  int* err;
  long long ncol, NxNy, plane, chan;  // columns B Nx Ny; points per column; per channel
  int Ci, Co, Nz, Nt, Jz, Jt, KT, KZ, NH, NCK, S;
  uint32_t stage_bytes, stage_bytes_tx, o_dz, o_gp, o_fz, o_bar;  // slot stride; bytes copied per chunk
};

// Byte offset of (row r, block b, point p) in a staged box whose start is
// 1024-byte aligned: line 9 r + b, its 16-byte chunks permuted by the line's
// XOR class (9 r + b) mod 8 = (r + b) mod 8.
__device__ __forceinline__ uint32_t swz(uint32_t r, uint32_t b, uint32_t p) {
  return r * kDtRow + b * 128u + ((((p >> 2) ^ (r + b)) & 7u) << 4) + (p & 3u) * 4u;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(c1), "r"(c2), "r"(tma::smem_u32(bar))
      : "memory");
}

// One bounded wait by the calling thread; also ends when the CTA aborts.  A
// waiting warp sleeps between tries so that it takes no issue slots from the
// warps that work.
__device__ __forceinline__ bool dt_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (tma::mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 8; ++i) {
      __nanosleep(64);
      if (tma::mbar_try_wait(bar, parity)) return true;
    }
    if (*abort_flag) return false;
    if (clock64() - t0 > kDtWait) return false;
  }
}
// The same for a whole warp, with a uniform result.
__device__ __forceinline__ bool dt_wait_warp(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  return __all_sync(0xffffffffu, dt_wait(bar, parity, abort_flag));
}

__device__ __forceinline__ void bar_a() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// barrier of the DFT warps (named barrier 2) that also ANDs a predicate, so
// that they take every decision to leave together
__device__ __forceinline__ bool bar_b_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, 2, 256, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}
}  // namespace

template <bool SPLIT, bool TF, int MZ>
__global__ void __launch_bounds__(kDtThreads, 1) k_da_tz(const __grid_constant__ DaTz p) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  // staged boxes start on 1024-byte boundaries (the swizzle repeats every 1024 bytes)
  const uint32_t raw = tma::smem_u32(dsm);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  unsigned char* sm = dsm + pad;
  const uint32_t sbase = raw + pad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g8 = lane >> 2, t4 = lane & 3;
  const int S = p.S;
  const int Ci = p.Ci, Co = p.Co, Nt = p.Nt;
  uint4* fzf = reinterpret_cast<uint4*>(sm + p.o_fz);  // [MZ][KZ][4 parts][32 lanes]
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + p.o_bar);  // [S] the chunk has landed
  uint64_t* dav = full + S;                                     // [S] its dA is in place
  int* left = reinterpret_cast<int*>(dav + S);                  // [S] warps not done with the chunk
  volatile int* abort_flag = left + S;
  int* s_issued = left + S + 1;                                 // chunks issued so far
  auto raise = [&]() {
    *abort_flag = 1;
    atomicExch(p.err, 1);
  };

  // z basis in A-fragment order: parts (re hi, re lo, im hi, im lo); rows kz,
  // cols z; a0 = (kz g8, z 2 t4 + {0,1}), a1 = (kz g8 + 8, ...), a2, a3 at z + 8
  for (int e = tid; e < MZ * p.KZ * 32; e += kDtThreads) {
    const int ln = e & 31, ks = (e >> 5) % p.KZ, mt = (e >> 5) / p.KZ;
    const int r0 = 16 * mt + (ln >> 2), c0 = 16 * ks + 2 * (ln & 3);
    auto F = [&](int kz, int z, int im) -> float {
      if (kz >= p.Jz || z >= p.Nz) return 0.f;
      const float2 f = p.Fz[(long long)kz * p.Nz + z];
      return wm::rnd<TF>(im ? f.y : f.x);
    };
#pragma unroll
    for (int im = 0; im < 2; ++im) {
      uint32_t h[4], l[4];
      wm::split2(F(r0, c0, im), F(r0, c0 + 1, im), h[0], l[0]);
      wm::split2(F(r0 + 8, c0, im), F(r0 + 8, c0 + 1, im), h[1], l[1]);
      wm::split2(F(r0, c0 + 8, im), F(r0, c0 + 9, im), h[2], l[2]);
      wm::split2(F(r0 + 8, c0 + 8, im), F(r0 + 8, c0 + 9, im), h[3], l[3]);
      const int base = ((mt * p.KZ + ks) * 4 + 2 * im) * 32 + ln;
      fzf[base] = make_uint4(h[0], h[1], h[2], h[3]);
      fzf[base + 32] = make_uint4(l[0], l[1], l[2], l[3]);
    }
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      tma::mbar_init(&full[s], 1);
      tma::mbar_init(&dav[s], kDtWarpsA);
      left[s] = kDtWarpsA + kDtWarpsB;
    }
    *abort_flag = 0;
    *s_issued = 0;
    tma::fence_mbar_init();
  }
  __syncthreads();

  const long long c_begin = p.ncol * blockIdx.x / gridDim.x;
  const long long c_end = p.ncol * (blockIdx.x + 1) / gridDim.x;
  const long long nst = (c_end - c_begin) * p.NCK;  // chunks of this CTA, in column order
  auto chunk_at = [&](long long g, long long& b, long long& xy, int& k) {
    const long long c = c_begin + g / p.NCK;
    k = (int)(g % p.NCK);
    b = c / p.NxNy;
    xy = c - b * p.NxNy;
  };
  // the coordinates of consecutive chunks, without divisions
  struct Walk {
    long long b, xy;
    int k;
  };
  auto walk_start = [&]() {
    Walk q;
    chunk_at(0, q.b, q.xy, q.k);
    return q;
  };
  auto walk_next = [&](Walk& q) {
    if (++q.k == p.NCK) {
      q.k = 0;
      if (++q.xy == p.NxNy) {
        q.xy = 0;
        ++q.b;
      }
    }
  };
  // Chunk g goes into slot g % S: the first S chunks now, by thread 0; chunk
  // g + S by the warp that finishes chunk g last (release_slot).
  // (32-bit arithmetic: the host keeps chunk and block counts below 2^31)
  const int cb32 = (int)c_begin, nck = p.NCK, nxny = (int)p.NxNy, bpc = (int)(p.plane >> 5);
  auto issue = [&](int g, int s) {
    const int cl = g / nck, k = g - cl * nck, c = cb32 + cl;
    const int b = c / nxny, xy = c - b * nxny;
    const int blk0 = xy * bpc + k * (kDtPoints / 32);
    const uint32_t st = sbase + (uint32_t)s * p.stage_bytes;
    tma::fence_proxy_async();
    tma::mbar_arrive_expect_tx(&full[s], p.stage_bytes_tx);
    tma_load_3d(st, &p.mx, blk0, b * Ci, &full[s]);
    tma_load_3d(st + p.o_dz, &p.mdz, blk0, b * Co, &full[s]);
    tma_load_3d(st + p.o_gp, &p.mgp, blk0, b * Co, &full[s]);
    atomicMax(s_issued, g + 1);
  };
  if (tid == 0)
    for (int g = 0; g < S && g < nst; ++g) issue(g, g);
  // this warp is done with chunk g (slot s): the last of the sixteen refills the slot
  auto release_slot = [&](long long g, int s) {
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      if (atomicSub(&left[s], 1) == 1) {
        __threadfence_block();
        left[s] = kDtWarpsA + kDtWarpsB;
        if (g + S < nst) issue((int)(g + S), s);
      }
    }
    __syncwarp();
  };

  if (warp < kDtWarpsA) {
    // ================= dW warps: (dW_lin, db) over block w ===================
    const int w = warp;
    const int MT = (Ci + 1 + 15) / 16, NT = (Co + 7) / 8;
    // Per-thread byte offsets in a staged box: every access below is one of
    // eight precomputed offsets plus a compile-time multiple of the row size.
    //   x rows g8 + 8 q', block w, points 8 kk + t4 (+4), and dA rows g8 + 8 n
    //   likewise                                  -> ofr[2 kk (+1)] + kDtRow 8 q'
    uint32_t ofr[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) ofr[j] = swz((uint32_t)g8, (uint32_t)w, (uint32_t)(4 * j + t4));
    float sum[2][3][4], cmp[2][3][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int n = 0; n < 3; ++n)
#pragma unroll
        for (int q = 0; q < 4; ++q) sum[m][n][q] = cmp[m][n][q] = 0.f;
    // x fragment rows i = 16 m + g8 + 8 r: loaded (i < Ci), the ones row (i == Ci) or zero
    bool xin[2][2];
    float xone[2][2];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int i = 16 * m + g8 + 8 * r;
        xin[m][r] = i < Ci;
        xone[m][r] = (i == Ci) ? 1.f : 0.f;
      }
    const bool din[3] = {g8 < Co, 8 + g8 < Co, 16 + g8 < Co};
    int s = 0;
    uint32_t ph = 0;
    for (long long g = 0; g < nst; ++g, s = (s + 1 == S) ? 0 : s + 1, ph ^= (s == 0)) {
      // the chunk has landed and the DFT warps have put dA in place of dz
      if (!dt_wait_warp(&dav[s], ph, abort_flag)) {
        if (lane == 0) raise();
        break;
      }
      const unsigned char* xs = sm + (size_t)s * p.stage_bytes;
      const unsigned char* ds = sm + (size_t)s * p.stage_bytes + p.o_dz;
      // (dW_lin, db) over the 32 points of block w: rows i of x (row Ci the
      // ones row of db; rows past it enter as zeros), columns o of dA (columns
      // past Co are zeros and discarded), k = point
      float acc[2][3][4];
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[m][n][q] = 0.f;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        uint32_t ab[2][4], as[2][4];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          if (m < MT) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              float xv = xone[m][q & 1];
              if (xin[m][q & 1])
                xv = *reinterpret_cast<const float*>(xs + ofr[2 * kk + (q >> 1)] +
                                                     kDtRow * (uint32_t)(16 * m + 8 * (q & 1)));
              wm::tf32_split_int(xv, ab[m][q], as[m][q]);
            }
          }
        }
#pragma unroll
        for (int n = 0; n < 3; ++n) {
          if (n < NT) {
            float d0 = 0.f, d1 = 0.f;
            if (din[n]) {
              d0 = *reinterpret_cast<const float*>(ds + ofr[2 * kk] + kDtRow * (uint32_t)(8 * n));
              d1 = *reinterpret_cast<const float*>(ds + ofr[2 * kk + 1] + kDtRow * (uint32_t)(8 * n));
            }
            uint32_t bb0, bs0, bb1, bs1;
            wm::tf32_split_int(d0, bb0, bs0);
            wm::tf32_split_int(d1, bb1, bs1);
#pragma unroll
            for (int m = 0; m < 2; ++m) {
              if (m < MT) {
                wm::mma_tf32(acc[m][n], as[m], bb0, bb1);
                wm::mma_tf32(acc[m][n], ab[m], bs0, bs1);
                wm::mma_tf32(acc[m][n], ab[m], bb0, bb1);
              }
            }
          }
        }
      }
      release_slot(g, s);
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
          for (int q = 0; q < 4; ++q) {  // Kahan: sum - cmp tracks the exact total
            const float yv = acc[m][n][q] - cmp[m][n][q];
            const float tv = sum[m][n][q] + yv;
            cmp[m][n][q] = (tv - sum[m][n][q]) - yv;
            sum[m][n][q] = tv;
          }
    }
    // (dW_lin, db) partials: fold[warp][pair] in the ring once every role is
    // done with it and every copy started has landed, then a fixed-order sum
    // over the warps
    const int npair = Ci * Co + Co;
    __syncthreads();
    if (tid == 0) {
      const long long issued = *s_issued;
      for (long long q = (issued > S ? issued - S : 0); q < issued; ++q)
        (void)tma::mbar_wait(&full[q % S], (uint32_t)((q / S) & 1), kDtWait);
    }
    bar_a();
    float* fold = reinterpret_cast<float*>(sm);
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int n = 0; n < 3; ++n)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = 16 * m + g8 + 8 * (q >> 1), o = 8 * n + 2 * t4 + (q & 1);
          if (m < MT && n < NT && i <= Ci && o < Co)
            fold[w * npair + (i < Ci ? i * Co + o : Ci * Co + o)] = sum[m][n][q] - cmp[m][n][q];
        }
    bar_a();
    for (int e = tid; e < npair; e += 32 * kDtWarpsA) {
      float sv = 0.f, cc = 0.f;
      for (int ww = 0; ww < kDtWarpsA; ++ww) {
        const float yv = fold[ww * npair + e] - cc;
        const float tv = sv + yv;
        cc = (tv - sv) - yv;
        sv = tv;
      }
      p.part[(long long)blockIdx.x * npair + e] = sv;
    }
    return;
  }

  // ================= DFT warps: dA, then the t, z DFT of dA ==================
  const int v = warp - kDtWarpsA;
  // t basis fragments in registers (KT <= 2): rows ri * 8 + jt, k slots
  // 2 t4 + {0,1} <-> t = 16 ks + 4 t4 + {0,1} and 2 t4 + 8 + {0,1} <-> + {2,3}
  uint4 frh[2], frl[2];
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    const int t0 = 16 * ks + 4 * t4;
    auto F = [&](int ri, int t) -> float {
      if (g8 >= p.Jt || t >= Nt || ks >= p.KT) return 0.f;
      const float2 f = p.Ft[(long long)g8 * Nt + t];
      return wm::rnd<TF>(ri ? f.y : f.x);
    };
    uint32_t h[4], l[4];
    wm::split2(F(0, t0), F(0, t0 + 1), h[0], l[0]);
    wm::split2(F(1, t0), F(1, t0 + 1), h[1], l[1]);
    wm::split2(F(0, t0 + 2), F(0, t0 + 3), h[2], l[2]);
    wm::split2(F(1, t0 + 2), F(1, t0 + 3), h[3], l[3]);
    frh[ks] = make_uint4(h[0], h[1], h[2], h[3]);
    frl[ks] = make_uint4(l[0], l[1], l[2], l[3]);
  }
  // the t stage reads channel o = v + 8 j at point (8 h + g8) Nt + 16 ks + 4 t4
  // of the chunk: otz[h][ks] + 8 kDtRow j (the XOR class of row o is that of v)
  uint32_t otz[2][2];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const uint32_t pt = (uint32_t)((8 * h + g8) * Nt + 16 * ks + 4 * t4) & 255u;
      otz[h][ks] = swz((uint32_t)v, pt >> 5, pt & 31u);
    }
  // the dA pass reads row o, block v, point lane: oda[o mod 8] + kDtRow (o - o mod 8)
  uint32_t oda[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) oda[j] = swz((uint32_t)j, (uint32_t)v, (uint32_t)lane);
  float tre[kDtCPW][MZ][4], tim[kDtCPW][MZ][4];
  uint32_t pend[kDtCPW][4];
#pragma unroll
  for (int j = 0; j < kDtCPW; ++j) {
#pragma unroll
    for (int mt = 0; mt < MZ; ++mt)
#pragma unroll
      for (int q = 0; q < 4; ++q) tre[j][mt][q] = tim[j][mt][q] = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) pend[j][q] = 0u;
  }
  Walk cw = walk_start();
  int s = 0;
  uint32_t ph = 0;
  for (long long g = 0; g < nst; ++g, walk_next(cw), s = (s + 1 == S) ? 0 : s + 1, ph ^= (s == 0)) {
    bool ok = dt_wait_warp(&full[s], ph, abort_flag);
    if (!ok && lane == 0) raise();
    const long long b = cw.b, xy = cw.xy;
    const int k = cw.k;
    unsigned char* db_ = sm + (size_t)s * p.stage_bytes + p.o_dz;
    if (ok) {
      // dA = dz GELU'(A) at the points 32 v .. 32 v + 31, in place and to global memory
      const unsigned char* gs = sm + (size_t)s * p.stage_bytes + p.o_gp;
      float* dag = p.da + (b * Co) * p.chan + xy * p.plane + (long long)k * kDtPoints + 32 * v + lane;
#pragma unroll
      for (int o = 0; o < kDtWarpsB * kDtCPW; ++o) {
        if (o < Co) {
          const uint32_t off = oda[o & 7] + kDtRow * (uint32_t)(o & ~7);
          float* dp = reinterpret_cast<float*>(db_ + off);
          const float dv = *dp * *reinterpret_cast<const float*>(gs + off);
          *dp = dv;
          dag[(long long)o * p.chan] = dv;
        }
      }
      __syncwarp();
      if (lane == 0) tma::mbar_arrive(&dav[s]);
    }
    // every DFT warp's dA is in place (the t stage reads every block); the
    // DFT warps take every decision to leave together
    if (!bar_b_and(ok && *abort_flag == 0)) break;
#pragma unroll
    for (int j = 0; j < kDtCPW; ++j) {
      const int o = v + kDtWarpsB * j;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (o >= Co || h >= p.NH) continue;  // uniform over the warp
        const int hz = k * p.NH + h;
        float pc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          if (ks >= p.KT) continue;
          const float4 x4 = *reinterpret_cast<const float4*>(db_ + otz[h][ks] + 8u * kDtRow * (uint32_t)j);
          uint32_t bh0, bl0, bh1, bl1;
          wm::split2(wm::rnd<TF>(x4.x), wm::rnd<TF>(x4.y), bh0, bl0);
          wm::split2(wm::rnd<TF>(x4.z), wm::rnd<TF>(x4.w), bh1, bl1);
          if (SPLIT) {
            wm::mma16(pc, frl[ks].x, frl[ks].y, frl[ks].z, frl[ks].w, bh0, bh1);
            wm::mma16(pc, frh[ks].x, frh[ks].y, frh[ks].z, frh[ks].w, bl0, bl1);
          }
          wm::mma16(pc, frh[ks].x, frh[ks].y, frh[ks].z, frh[ks].w, bh0, bh1);
        }
        uint32_t rh, rl, ih, il;
        wm::split2(wm::rnd<TF>(pc[0]), wm::rnd<TF>(pc[1]), rh, rl);  // P_re at z, z + 1
        wm::split2(wm::rnd<TF>(pc[2]), wm::rnd<TF>(pc[3]), ih, il);  // P_im
        if ((hz & 1) == 0) {
          pend[j][0] = rh;
          pend[j][1] = rl;
          pend[j][2] = ih;
          pend[j][3] = il;
        } else {
          // z stage k-step kz: B = (planes 0..7 from the pending n-tile, 8..15 now)
          const int kz = hz >> 1;
          const uint32_t rh0 = pend[j][0], rl0 = pend[j][1], ih0 = pend[j][2], il0 = pend[j][3];
          const uint32_t nh0 = ih0 ^ 0x80008000u, nh1 = ih ^ 0x80008000u;  // -P_im
          const uint32_t nl0 = il0 ^ 0x80008000u, nl1 = il ^ 0x80008000u;
#pragma unroll
          for (int mt = 0; mt < MZ; ++mt) {
            const int base = ((mt * p.KZ + kz) * 4) * 32 + lane;
            const uint4 arh = fzf[base], arl = fzf[base + 32];
            const uint4 aih = fzf[base + 64], ail = fzf[base + 96];
            float dr[4] = {0.f, 0.f, 0.f, 0.f}, di[4] = {0.f, 0.f, 0.f, 0.f};
            if (SPLIT) {
              wm::mma16(dr, arl.x, arl.y, arl.z, arl.w, rh0, rh);
              wm::mma16(dr, arh.x, arh.y, arh.z, arh.w, rl0, rl);
              wm::mma16(dr, ail.x, ail.y, ail.z, ail.w, nh0, nh1);
              wm::mma16(dr, aih.x, aih.y, aih.z, aih.w, nl0, nl1);
              wm::mma16(di, arl.x, arl.y, arl.z, arl.w, ih0, ih);
              wm::mma16(di, arh.x, arh.y, arh.z, arh.w, il0, il);
              wm::mma16(di, ail.x, ail.y, ail.z, ail.w, rh0, rh);
              wm::mma16(di, aih.x, aih.y, aih.z, aih.w, rl0, rl);
            }
            wm::mma16(dr, arh.x, arh.y, arh.z, arh.w, rh0, rh);
            wm::mma16(dr, aih.x, aih.y, aih.z, aih.w, nh0, nh1);
            wm::mma16(di, arh.x, arh.y, arh.z, arh.w, ih0, ih);
            wm::mma16(di, aih.x, aih.y, aih.z, aih.w, rh0, rh);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              tre[j][mt][q] += dr[q];
              tim[j][mt][q] += di[q];
            }
          }
        }
      }
    }
    release_slot(g, s);
    if (k == p.NCK - 1) {
      // the column's spectrum: T[col][kz][jt], rows kz = 16 mt + g8 (+8), cols jt = 2 t4 + {0, 1}
#pragma unroll
      for (int j = 0; j < kDtCPW; ++j) {
        const int o = v + kDtWarpsB * j;
        if (o < Co) {
          float2* oc = p.out + ((b * Co + o) * p.NxNy + xy) * (long long)(p.Jz * p.Jt);
#pragma unroll
          for (int mt = 0; mt < MZ; ++mt)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              const int kz = 16 * mt + g8 + 8 * hh;
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const int jt = 2 * t4 + e;
                if (kz < p.Jz && jt < p.Jt)
                  oc[kz * p.Jt + jt] = make_float2(tre[j][mt][2 * hh + e], tim[j][mt][2 * hh + e]);
              }
            }
        }
#pragma unroll
        for (int mt = 0; mt < MZ; ++mt)
#pragma unroll
          for (int q = 0; q < 4; ++q) tre[j][mt][q] = tim[j][mt][q] = 0.f;
      }
    }
  }
  __syncthreads();  // pairs with the dW warps' barrier before their fold
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
cudaError_t encode_tiled(CUtensorMap* map, const void* base, int rank, const cuuint64_t* dims,
                         const cuuint64_t* strides, const cuuint32_t* box, bool swizzle128);

static constexpr size_t kDtSmemMax = 227 * 1024;
static uint32_t al1024(uint32_t x) { return (x + 1023u) & ~1023u; }

// Shapes and the shared-memory plan: chunks of 256 points are whole z-planes
// (Nt 16 or 32) that pair into 16-plane z k-steps (Nz a multiple of 16); the
// (dW_lin, db) fragments cover C_in + 1 <= 32 rows and C_out <= 24 columns;
// the t basis stays in registers (Jt <= 8, two k-steps), the z basis in
// shared memory (Jz <= 32).  A slot holds the x, dz and GELU'(A) boxes, each
// starting on a 1024-byte boundary.
static bool da_tz_plan(const Dims& d, DaTz& k, size_t& smem, const char** why) {
  const char* r = nullptr;
  if (d.Nt != 16 && d.Nt != 32) r = "Nt is not 16 or 32";
  else if (d.Nz % 16 != 0) r = "Nz is not a multiple of 16";
  else if (d.Jt > 8) r = "more than 8 kept t modes";
  else if (d.Jz > 32) r = "more than 32 kept z modes";
  else if (d.Ci + 1 > 32 || d.Co > kDtWarpsB * kDtCPW) r = "more than 31 input or 24 output channels";
  else if (d.B * d.Ci > (1 << 30) || d.B * d.Co > (1 << 30) || d.Ng / 32 > (1LL << 30) ||
           d.B * d.Nx * d.Ny * (d.Nz * d.Nt / kDtPoints) > (1LL << 30))
    r = "sizes too large";
  if (r) {
    if (why) *why = r;
    return false;
  }
  k.Ci = (int)d.Ci;
  k.Co = (int)d.Co;
  k.Nz = (int)d.Nz;
  k.Nt = (int)d.Nt;
  k.Jz = (int)d.Jz;
  k.Jt = (int)d.Jt;
  k.KT = (int)(d.Nt / 16);
  k.KZ = (int)(d.Nz / 16);
  k.NH = kDtPoints / k.Nt / 8;
  k.NCK = k.Nz / (kDtPoints / k.Nt);
  k.NxNy = d.Nx * d.Ny;
  k.plane = d.Nz * d.Nt;
  k.chan = d.Ng;
  k.ncol = d.B * k.NxNy;
  const int MZ = (k.Jz + 15) / 16;
  k.o_dz = al1024(kDtRow * (uint32_t)k.Ci);
  k.o_gp = k.o_dz + al1024(kDtRow * (uint32_t)k.Co);
  k.stage_bytes = k.o_gp + al1024(kDtRow * (uint32_t)k.Co);
  k.stage_bytes_tx = kDtRow * (uint32_t)(k.Ci + 2 * k.Co);
  const uint32_t fz_bytes = (uint32_t)MZ * (uint32_t)k.KZ * 2048u;
  for (int S = 4; S >= 2; --S) {
    const uint32_t o_fz = (uint32_t)S * k.stage_bytes;
    const uint32_t o_bar = o_fz + fz_bytes;
    const size_t total = (size_t)o_bar + 16u * (uint32_t)S + 4u * (uint32_t)(S + 2) + 1024u;  // + alignment pad
    if (total <= kDtSmemMax) {
      k.S = S;
      k.o_fz = o_fz;
      k.o_bar = o_bar;
      smem = total;
      return true;
    }
  }
  if (why) *why = "the staging ring does not fit in shared memory";
  return false;
}

// [rows][blocks of 32 points][32 points] view of a [rows][chan] FP32 array;
// boxes of box_rows x 9 blocks x 32 points with the 128-byte swizzle (a box may
// reach one block past the end of a row: the copy fills it with zeros)
static cudaError_t encode_blocked_map(CUtensorMap* map, const float* base, long long chan, long long rows,
                                      int box_rows) {
  const cuuint64_t dims[3] = {32u, (cuuint64_t)(chan / 32), (cuuint64_t)rows};
  const cuuint64_t strides[2] = {128u, (cuuint64_t)chan * sizeof(float)};
  const cuuint32_t box[3] = {32u, (cuuint32_t)kDtBoxBlocks, (cuuint32_t)box_rows};
  return encode_tiled(map, base, 3, dims, strides, box, true);
}

bool da_tz_supported(const Dims& d, char* why, size_t nwhy) {
  DaTz k{};
  size_t smem = 0;
  const char* r = nullptr;
  bool ok = da_tz_plan(d, k, smem, &r);
  if (ok) {
    // the blocked, swizzled tensor maps must encode for these sizes (host only)
    CUtensorMap m;
    const float* probe = reinterpret_cast<const float*>(256);
    if (encode_blocked_map(&m, probe, d.Ng, d.B * d.Ci, (int)d.Ci) != cudaSuccess ||
        encode_blocked_map(&m, probe, d.Ng, d.B * d.Co, (int)d.Co) != cudaSuccess) {
      r = "the tensor maps of the blocked layout do not encode";
      ok = false;
    }
  }
  if (!ok && why) snprintf(why, nwhy, "%s", r);
  return ok;
}

template <bool SPLIT, bool TF, int MZ>
static cudaError_t launch_da_tz_t(const DaTz& k, size_t smem, int grid, const char* name, cudaStream_t s) {
  cudaError_t e =
      cudaFuncSetAttribute(k_da_tz<SPLIT, TF, MZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  FNO_LAUNCH(name, (k_da_tz<SPLIT, TF, MZ>), grid, kDtThreads, smem, s, k);
  return cudaSuccess;
}

template <int MZ>
static cudaError_t launch_da_tz_m(const DaTz& k, size_t smem, int grid, bool split, bool tf32, cudaStream_t s) {
  if (tf32) return launch_da_tz_t<true, true, MZ>(k, smem, grid, "fno_da_tz_tf32", s);
  if (split) return launch_da_tz_t<true, false, MZ>(k, smem, grid, "fno_da_tz_bf16x3", s);
  return launch_da_tz_t<false, false, MZ>(k, smem, grid, "fno_da_tz_bf16", s);
}

cudaError_t launch_da_tz(const float* x, const float* g, const float* dz, float* da, float2* t1, float* part,
                         int max_rows, const Dims& d, const float2* ft, const float2* fz, bool split, bool tf32,
                         int* err, int* rows_out, cudaStream_t s) {
  DaTz k{};
  size_t smem = 0;
  const char* why = nullptr;
  if (!da_tz_plan(d, k, smem, &why)) return cudaErrorInvalidValue;
  cudaError_t e = encode_blocked_map(&k.mx, x, k.chan, d.B * d.Ci, (int)d.Ci);
  if (e == cudaSuccess) e = encode_blocked_map(&k.mdz, dz, k.chan, d.B * d.Co, (int)d.Co);
  if (e == cudaSuccess) e = encode_blocked_map(&k.mgp, g, k.chan, d.B * d.Co, (int)d.Co);
  if (e != cudaSuccess) return e;
  k.Ft = ft;
  k.Fz = fz;
  k.da = da;
  k.out = t1;
  k.part = part;
  k.err = err;
  const int grid = (int)std::max<long long>(1, std::min<long long>({(long long)sm_count(), k.ncol, (long long)max_rows}));
  *rows_out = grid;
  if (k.Jz <= 16) return launch_da_tz_m<1>(k, smem, grid, split, tf32, s);
  return launch_da_tz_m<2>(k, smem, grid, split, tf32, s);
}

}  // namespace fno
