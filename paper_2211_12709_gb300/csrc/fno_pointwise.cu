// fno_pointwise.cu -- the layers around the FNO blocks in Alg. 1 (Sec. IV-C):
// the encoder and decoder 1x1 convolutions with sigma, and the training loss.
//
//   forward   y[b,o,p] = act(A),  A = sum_i x[b,i,p] w[i,o] + bias[o]
//   backward  dA = dy act'(A);  dx[b,i,p] = sum_o w[i,o] dA[b,o,p]
//             dw[i,o] = sum_{b,p} x[b,i,p] dA[b,o,p];  db[o] = sum_{b,p} dA[b,o,p]
//   loss      L = (1/n) sum (y - t)^2;  dy = (2/n) (y - t)
//
// These layers have few channels on one side (the CO2 model lifts 3 input
// channels to width 20 and projects 20 to 1), so they move a few bytes per
// multiply-add and are bound by HBM: FP32 on the CUDA cores, no tensor cores.
//
// sigma is GELU with erf from Abramowitz and Stegun 7.1.26 (|error| < 1.5e-7).
//
// Forward: each thread owns 4 consecutive points (16-byte loads and stores)
// and writes their C_out outputs, taking the weights from shared memory.
//
// Backward: a persistent CTA walks 256-point tiles of one batch entry.  The
// tile's rows of x and dy are staged in shared memory by cp.async: 16-byte
// copies when the rows are 16-byte aligned (P a multiple of 4), 4-byte copies
// otherwise, zero-filled past the ragged end of a channel.  With room for two
// stages the next tile's copies are in flight while the current one is
// computed; otherwise a tile's copies are issued together and waited for once.
// Each thread forms dA for its point in place and, when asked, dx
// for its point; then every thread accumulates a 2 x 4 block of the (input,
// output) pairs of dW over its share of the tile's points (a row of ones next
// to x gives db).  Per-tile sums are added into per-thread Kahan accumulators,
// so each pair's error stays near one rounding per tile; at the end the CTA
// folds its threads in a fixed order and writes one row of partial sums, which
// launch_reduce_partials adds over CTAs, again in a fixed order.  Results are
// bitwise reproducible for a given device and sizes.
//
// Loss: grid-stride pass writing dy with per-thread Kahan sums of (y - t)^2,
// a fixed-order block reduction to one partial per CTA, and a one-CTA final sum.
//
// Training step: an in-place Adam update of one parameter tensor.
//
// The block backward after a training forward uses the same staging for its
// dA pass: dA = dz GELU'(A) from the forward's saved GELU'(A), written out,
// with the (dW_lin, db) partial sums.  Up to 31 inputs and 24 outputs that
// contraction runs on the tensor cores (k_da_mma, split TF32 products);
// wider layers take the pair blocks of k_pw_bwd.
#include <algorithm>

#include "fno_internal.h"
#include "warp_mma.h"

namespace fno {

namespace {

constexpr int kPwThreads = 256;
constexpr int kPwTile = 256;         // points per tile
constexpr int kPwLd = kPwTile + 4;   // row stride of a staged tile (16-byte rows)
constexpr int kPwOc = 8;             // output channels per register chunk
constexpr size_t kPwTwoStageMax = 100 * 1024;  // stage bytes up to which tiles double-buffer

struct PwArgs {
  const float* x;
  const float* w;
  const float* bias;  // nullable
  const float* dy;
  const float* gs;    // nullable: saved act'(A) [B][Co][P] (block backward after a training forward)
  float* da;          // with gs: dA = dy * gs written here [B][Co][P]
  float* y;           // forward output
  float* dx;          // nullable
  float* part;        // [grid][npair] partial sums of (dw, db)
  long long B, P;
  int Ci, Co, act, nstage;
};

__device__ __forceinline__ float act_f(float a, int act) { return act ? gelu_as(a) : a; }

__device__ __forceinline__ uint32_t pw_smem(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// asynchronous global -> shared copies; bytes < size zero-fills the rest
__device__ __forceinline__ void cp_async16(float* dst, const float* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(pw_smem(dst)), "l"(src),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(pw_smem(dst)), "l"(src),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Stage rows [0, rows) of a tile: row r starts at src + r * P + p0 and holds np
// valid points; dst is [rows][kPwLd].  VEC needs P % 4 == 0 and 16-byte src.
template <bool VEC>
__device__ __forceinline__ void stage_rows(float* dst, const float* src, int rows, long long P,
                                           long long p0, int np) {
  if (VEC) {
    constexpr int G = kPwTile / 4;
    for (int e = threadIdx.x; e < rows * G; e += kPwThreads) {
      const int r = e / G, c = (e - r * G) * 4;
      const bool ok = c < np;  // np is a multiple of 4 here
      cp_async16(dst + r * kPwLd + c, src + r * P + p0 + (ok ? c : 0), ok ? 16 : 0);
    }
  } else {
    for (int e = threadIdx.x; e < rows * kPwTile; e += kPwThreads) {
      const int r = e / kPwTile, c = e - r * kPwTile;
      const bool ok = c < np;
      cp_async4(dst + r * kPwLd + c, src + r * P + p0 + (ok ? c : 0), ok ? 4 : 0);
    }
  }
}

struct TileOf {
  long long b, p0;
  int np;
};
__device__ __forceinline__ TileOf tile_of(long long tile, long long tpb, long long P) {
  TileOf t;
  // tile < 2^32 for every realistic size: a 32-bit division is far cheaper
  t.b = (tile < 0xffffffffLL) ? (long long)((unsigned)tile / (unsigned)tpb) : tile / tpb;
  t.p0 = (tile - t.b * tpb) * kPwTile;
  const long long left = P - t.p0;
  t.np = (int)(left < kPwTile ? left : kPwTile);
  return t;
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
// Each thread owns V consecutive points (V = 4: 16-byte loads and stores, when
// P is a multiple of 4 and the tensors 16-byte aligned) and walks the outputs
// in chunks of 8; its x values are reloaded per chunk (L1 hits after the
// first).  The input loop is unrolled by 4 so that several loads are in flight.
template <int V>
__global__ void __launch_bounds__(kPwThreads) k_pw_fwd(const PwArgs k) {
  extern __shared__ float sm[];
  float* ws = sm;                    // [Ci][Co]
  float* bs = sm + k.Ci * k.Co;      // [Co]
  for (int e = threadIdx.x; e < k.Ci * k.Co; e += blockDim.x) ws[e] = k.w[e];
  for (int e = threadIdx.x; e < k.Co; e += blockDim.x) bs[e] = k.bias ? k.bias[e] : 0.f;
  __syncthreads();
  const long long groups = (k.P + V - 1) / V;  // V divides P when V > 1
  const long long items = k.B * groups;
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const long long b = (it < 0xffffffffLL && groups < 0xffffffffLL)
                            ? (long long)((unsigned)it / (unsigned)groups) : it / groups;
    const long long p = (it - b * groups) * V;
    const float* xb = k.x + b * k.Ci * k.P + p;
    float* yb = k.y + b * k.Co * k.P + p;
    if (k.Co == 1) {  // one output (a decoder to one channel): no channel chunk
      float acc[V];
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = bs[0];
#pragma unroll 4
      for (int i = 0; i < k.Ci; ++i) {
        const float wv = ws[i];
        if (V == 4) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(xb + (long long)i * k.P));
          acc[0] = fmaf(q.x, wv, acc[0]);
          acc[V > 1 ? 1 : 0] = fmaf(q.y, wv, acc[V > 1 ? 1 : 0]);
          acc[V > 2 ? 2 : 0] = fmaf(q.z, wv, acc[V > 2 ? 2 : 0]);
          acc[V > 3 ? 3 : 0] = fmaf(q.w, wv, acc[V > 3 ? 3 : 0]);
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v] = fmaf(__ldg(xb + (long long)i * k.P + v), wv, acc[v]);
        }
      }
      if (V == 4) {
        float4 q;
        q.x = act_f(acc[0], k.act);
        q.y = act_f(acc[V > 1 ? 1 : 0], k.act);
        q.z = act_f(acc[V > 2 ? 2 : 0], k.act);
        q.w = act_f(acc[V > 3 ? 3 : 0], k.act);
        *reinterpret_cast<float4*>(yb) = q;
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) yb[v] = act_f(acc[v], k.act);
      }
      continue;
    }
    for (int o0 = 0; o0 < k.Co; o0 += kPwOc) {
      float acc[kPwOc][V];
#pragma unroll
      for (int c = 0; c < kPwOc; ++c) {
        const float bv = (o0 + c < k.Co) ? bs[o0 + c] : 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) acc[c][v] = bv;
      }
#pragma unroll 4
      for (int i = 0; i < k.Ci; ++i) {
        float xv[V];
        if (V == 4) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(xb + (long long)i * k.P));
          xv[0] = q.x;
          xv[V > 1 ? 1 : 0] = q.y;
          xv[V > 2 ? 2 : 0] = q.z;
          xv[V > 3 ? 3 : 0] = q.w;
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v) xv[v] = __ldg(xb + (long long)i * k.P + v);
        }
        const float* wr = ws + i * k.Co + o0;
#pragma unroll
        for (int c = 0; c < kPwOc; ++c) {
          const float wv = (o0 + c < k.Co) ? wr[c] : 0.f;
#pragma unroll
          for (int v = 0; v < V; ++v) acc[c][v] = fmaf(xv[v], wv, acc[c][v]);
        }
      }
#pragma unroll
      for (int c = 0; c < kPwOc; ++c) {
        if (o0 + c >= k.Co) break;
        float* dst = yb + (long long)(o0 + c) * k.P;
        if (V == 4) {
          float4 q;
          q.x = act_f(acc[c][0], k.act);
          q.y = act_f(acc[c][V > 1 ? 1 : 0], k.act);
          q.z = act_f(acc[c][V > 2 ? 2 : 0], k.act);
          q.w = act_f(acc[c][V > 3 ? 3 : 0], k.act);
          *reinterpret_cast<float4*>(dst) = q;
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v) dst[v] = act_f(acc[c][v], k.act);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------
// Pair blocks: inputs i in [0, Ci] (i = Ci is the row of ones that gives db) in
// pairs, outputs in fours (inputs in eights when C_out = 1): nblk = ceil((Ci +
// 1) / 2) * ceil(Co / 4), or ceil((Ci + 1) / 8).  With
// nblk <= 256 the tile's points are split into S = 256 / nblk interleaved
// segments (thread -> block tid % nblk, segment tid / nblk); otherwise S = 1
// and each thread owns up to KB blocks (tid, tid + 256, ...).
struct PwPlan {
  int nbi, nbo, nblk, S, KB, npair, nstage;
  size_t smem;  // bytes
};

// gs: the tiles also stage the saved derivative (C_out more rows)
PwPlan pw_plan(int Ci, int Co, bool gs = false) {
  PwPlan pl{};
  // blocks of 2 inputs x 4 outputs; 8 inputs x 1 output when C_out = 1
  pl.nbi = (Co == 1) ? (Ci + 8) / 8 : (Ci + 2) / 2;
  pl.nbo = (Co == 1) ? 1 : (Co + 3) / 4;
  pl.nblk = pl.nbi * pl.nbo;
  pl.S = pl.nblk <= kPwThreads ? kPwThreads / pl.nblk : 1;
  pl.KB = (pl.nblk + kPwThreads - 1) / kPwThreads;
  pl.npair = Ci * Co + Co;
  const size_t stage = sizeof(float) * (size_t)(Ci + 1 + Co + (gs ? Co : 0)) * kPwLd;
  pl.nstage = stage <= kPwTwoStageMax ? 2 : 1;
  const size_t stages = pl.nstage * stage;
  const size_t fold = sizeof(float) * (size_t)pl.S * pl.npair;
  pl.smem = std::max(stages, fold) + sizeof(float) * ((size_t)Ci * Co + Co);
  return pl;
}

template <int KB, bool VEC>
__global__ void __launch_bounds__(kPwThreads, KB == 1 ? 4 : 1) k_pw_bwd(const PwArgs k, const int nbo,
                                                       const int nblk, const int S,
                                                       const size_t stage_floats) {
  extern __shared__ __align__(16) float sm[];
  const int Ci = k.Ci, Co = k.Co;
  const int npair = Ci * Co + Co;
  const int RS = Ci + 1 + Co + (k.gs ? Co : 0);       // rows per stage
  float* stage = sm;                                   // [nstage][RS][kPwLd]
  float* fold = sm;                                    // reused at the end: [S][npair]
  float* ws = sm + stage_floats;                       // [Ci][Co]
  float* bs = ws + Ci * Co;                            // [Co]
  const int tid = threadIdx.x;
  for (int e = tid; e < Ci * Co; e += kPwThreads) ws[e] = k.w ? k.w[e] : 0.f;
  for (int e = tid; e < Co; e += kPwThreads) bs[e] = k.bias ? k.bias[e] : 0.f;

  // this thread's pair blocks
  const int seg = (nblk <= kPwThreads) ? tid / nblk : 0;
  const bool active = (nblk <= kPwThreads) ? (tid < nblk * S) : true;
  float sum[KB][8], comp[KB][8];
#pragma unroll
  for (int q = 0; q < KB; ++q)
#pragma unroll
    for (int e = 0; e < 8; ++e) sum[q][e] = comp[q][e] = 0.f;

  const long long tpb = (k.P + kPwTile - 1) / kPwTile;
  const long long ntiles = k.B * tpb;
  auto issue = [&](long long tl, int st) {
    const TileOf q = tile_of(tl, tpb, k.P);
    float* xs = stage + st * RS * kPwLd;
    stage_rows<VEC>(xs, k.x + q.b * Ci * k.P, Ci, k.P, q.p0, q.np);
    stage_rows<VEC>(xs + (Ci + 1) * kPwLd, k.dy + q.b * Co * k.P, Co, k.P, q.p0, q.np);
    if (k.gs) stage_rows<VEC>(xs + (Ci + 1 + Co) * kPwLd, k.gs + q.b * Co * k.P, Co, k.P, q.p0, q.np);
    cp_async_commit();
  };
  long long tile = blockIdx.x;
  if (tile < ntiles) issue(tile, 0);
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const int st = (k.nstage == 2) ? (it & 1) : 0;
    const long long nxt = tile + gridDim.x;
    if (k.nstage == 2 && nxt < ntiles) {
      issue(nxt, st ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // every thread's copies of this tile have landed
    const TileOf q = tile_of(tile, tpb, k.P);
    const int np = q.np;
    float* xs = stage + st * RS * kPwLd;   // [Ci + 1][kPwLd]  (row Ci = ones)
    float* ds = xs + (Ci + 1) * kPwLd;     // [Co][kPwLd]      dy, then dA
    {
      const int t = tid;
      const bool in = t < np;
      xs[Ci * kPwLd + t] = in ? 1.f : 0.f;
      // dA for this thread's point (its own column only: no barrier needed)
      if (k.gs && in) {  // dA = dy * saved act'(A), kept in the tile and written out
        const float* gr = ds + Co * kPwLd;
        float* dout = k.da + (q.b * Co) * k.P + q.p0 + t;
#pragma unroll 4
        for (int o = 0; o < Co; ++o) {
          const float v = ds[o * kPwLd + t] * gr[o * kPwLd + t];
          ds[o * kPwLd + t] = v;
          dout[(long long)o * k.P] = v;
        }
      } else if (k.act && in && Co == 1) {  // one output: no channel chunk
        float a0 = bs[0];
#pragma unroll 4
        for (int i = 0; i < Ci; ++i) a0 = fmaf(xs[i * kPwLd + t], ws[i], a0);
        ds[t] *= gelu_grad_as(a0);
      } else if (k.act && in) {
        for (int o0 = 0; o0 < Co; o0 += kPwOc) {
          float a[kPwOc];
#pragma unroll
          for (int c = 0; c < kPwOc; ++c) a[c] = (o0 + c < Co) ? bs[o0 + c] : 0.f;
          for (int i = 0; i < Ci; ++i) {
            const float xv = xs[i * kPwLd + t];
            const float* wr = ws + i * Co + o0;
#pragma unroll
            for (int c = 0; c < kPwOc; ++c)
              if (o0 + c < Co) a[c] = fmaf(xv, wr[c], a[c]);
          }
#pragma unroll
          for (int c = 0; c < kPwOc; ++c)
            if (o0 + c < Co) ds[(o0 + c) * kPwLd + t] *= gelu_grad_as(a[c]);
        }
      }
      if (k.dx && in) {
        for (int i0 = 0; i0 < Ci; i0 += kPwOc) {
          float g[kPwOc];
#pragma unroll
          for (int c = 0; c < kPwOc; ++c) g[c] = 0.f;
          for (int o = 0; o < Co; ++o) {
            const float dv = ds[o * kPwLd + t];
#pragma unroll
            for (int c = 0; c < kPwOc; ++c)
              if (i0 + c < Ci) g[c] = fmaf(ws[(i0 + c) * Co + o], dv, g[c]);
          }
#pragma unroll
          for (int c = 0; c < kPwOc; ++c)
            if (i0 + c < Ci) k.dx[(q.b * Ci + i0 + c) * k.P + q.p0 + t] = g[c];
        }
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int qb = 0; qb < KB; ++qb) {
        const int blk = (nblk <= kPwThreads) ? tid % nblk : tid + qb * kPwThreads;
        if (blk >= nblk) break;
        float acc[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[e] = 0.f;
        if (Co == 1) {  // 8 inputs x 1 output
          const int i0 = blk * 8;
          int xo[8];  // shared-memory row offsets (32-bit: fewer registers than pointers)
#pragma unroll
          for (int j = 0; j < 8; ++j) xo[j] = min(i0 + j, Ci) * kPwLd;
          for (int t = seg; t < np; t += S) {
            const float d0 = ds[t];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = fmaf(xs[xo[j] + t], d0, acc[j]);
          }
        } else {
        const int i0 = (blk / nbo) * 2, o0 = (blk % nbo) * 4;
        const float* xr0 = xs + i0 * kPwLd;
        const float* xr1 = xs + min(i0 + 1, Ci) * kPwLd;
        const float* dr0 = ds + min(o0 + 0, Co - 1) * kPwLd;
        const float* dr1 = ds + min(o0 + 1, Co - 1) * kPwLd;
        const float* dr2 = ds + min(o0 + 2, Co - 1) * kPwLd;
        const float* dr3 = ds + min(o0 + 3, Co - 1) * kPwLd;
        for (int t = seg; t < np; t += S) {
          const float x0 = xr0[t], x1 = xr1[t];
          const float d0 = dr0[t], d1 = dr1[t], d2 = dr2[t], d3 = dr3[t];
          acc[0] = fmaf(x0, d0, acc[0]);
          acc[1] = fmaf(x0, d1, acc[1]);
          acc[2] = fmaf(x0, d2, acc[2]);
          acc[3] = fmaf(x0, d3, acc[3]);
          acc[4] = fmaf(x1, d0, acc[4]);
          acc[5] = fmaf(x1, d1, acc[5]);
          acc[6] = fmaf(x1, d2, acc[6]);
          acc[7] = fmaf(x1, d3, acc[7]);
        }
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {  // Kahan: sum - comp tracks the exact total
          const float yv = acc[e] - comp[qb][e];
          const float tv = sum[qb][e] + yv;
          comp[qb][e] = (tv - sum[qb][e]) - yv;
          sum[qb][e] = tv;
        }
      }
    }
    __syncthreads();  // stage st is free for the copies issued next
    if (k.nstage == 1 && nxt < ntiles) issue(nxt, 0);
  }
  // fold this CTA's threads: fold[seg][pair], then a fixed-order sum per pair
  cp_async_wait<0>();
  __syncthreads();
  if (active) {
#pragma unroll
    for (int qb = 0; qb < KB; ++qb) {
      const int blk = (nblk <= kPwThreads) ? tid % nblk : tid + qb * kPwThreads;
      if (blk >= nblk) break;
      const bool one = (Co == 1);
      const int i0 = one ? blk * 8 : (blk / nbo) * 2, o0 = one ? 0 : (blk % nbo) * 4;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int i = one ? i0 + e : i0 + e / 4, o = one ? 0 : o0 + e % 4;
        if (i > Ci || o >= Co) continue;
        fold[seg * npair + i * Co + o] = sum[qb][e] - comp[qb][e];
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < npair; e += kPwThreads) {
    float s = 0.f, c = 0.f;
    for (int r = 0; r < S; ++r) {
      const float yv = fold[r * npair + e] - c;
      const float tv = s + yv;
      c = (tv - s) - yv;
      s = tv;
    }
    k.part[(long long)blockIdx.x * npair + e] = s;
  }
}

// ---------------------------------------------------------------------------
// dA pass of a block backward after a training forward, with dW_lin and db on
// the tensor cores, for C_in + 1 <= 32 rows and C_out <= 24
// ---------------------------------------------------------------------------
// A tile is 256 points of one batch entry: rows of x, a row of ones, dz and
// the saved GELU'(A), staged by cp.async.  Each thread forms dA = dz GELU'(A)
// for its point in place and writes it out; then warp w contracts points
// [32 w, 32 w + 32) of the tile:
//     acc[i][o] += sum_t X[i][t] dA[o][t]      (row i = C_in: the ones row, db)
// with warp-level mma.sync m16n8k8 on TF32 operands.  Each FP32 operand is
// split a = big + small (big = a rounded to TF32, small = the rest rounded to
// TF32) and three products big.big + big.small + small.big are summed, so a
// product carries about 2^-21 relative error, as FP32 would.  The fragments
// are read straight from the staged FP32 rows: with the row stride of 260
// floats the 32 lanes of a fragment load hit 32 different banks.  Per tile the
// products start from zero (short accumulation chains) and are Kahan-folded
// into per-thread sums; at the end the CTA adds its warps in a fixed order
// into one row of partial sums.
constexpr int kDaMT = 2;  // m-tiles of 16 over the C_in + 1 rows
constexpr int kDaNT = 3;  // n-tiles of 8 over the C_out columns

// a = big + small, both rounded to TF32 (nearest, ties away from zero; see
// warp_mma.h)
__device__ __forceinline__ void tf32_split(float a, uint32_t& big, uint32_t& small) {
  wm::tf32_split(a, big, small);
}
// D += A (16x8, row) * B (8x8, col), TF32 in, FP32 accumulate
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <bool VEC>
__global__ void __launch_bounds__(kPwThreads, 2) k_da_mma(const PwArgs k) {
  extern __shared__ __align__(16) float sm[];
  const int Ci = k.Ci, Co = k.Co;
  const int npair = Ci * Co + Co;
  const int RS = Ci + 1 + 2 * Co;   // rows per stage: x, ones, dz (then dA), GELU'(A)
  float* stage = sm;                 // [nstage][RS][kPwLd]
  float* fold = sm;                  // reused at the end: [8 warps][npair]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, c = lane & 3;
  const int MT = (Ci + 1 + 15) / 16, NT = (Co + 7) / 8;
  float sum[kDaMT][kDaNT][4], cmp[kDaMT][kDaNT][4];
#pragma unroll
  for (int m = 0; m < kDaMT; ++m)
#pragma unroll
    for (int n = 0; n < kDaNT; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) sum[m][n][q] = cmp[m][n][q] = 0.f;
  // fragment rows of x (clamped to the ones row; the extra rows are discarded)
  // and of dA (clamped to the last output; discarded likewise)
  int xr[kDaMT][2], dr[kDaNT];
#pragma unroll
  for (int m = 0; m < kDaMT; ++m) {
    xr[m][0] = min(16 * m + g, Ci) * kPwLd;
    xr[m][1] = min(16 * m + g + 8, Ci) * kPwLd;
  }
#pragma unroll
  for (int n = 0; n < kDaNT; ++n) dr[n] = min(8 * n + g, Co - 1) * kPwLd;

  const long long tpb = (k.P + kPwTile - 1) / kPwTile;
  const long long ntiles = k.B * tpb;
  auto issue = [&](long long tl, int st) {
    const TileOf q = tile_of(tl, tpb, k.P);
    float* xs = stage + st * RS * kPwLd;
    stage_rows<VEC>(xs, k.x + q.b * Ci * k.P, Ci, k.P, q.p0, q.np);
    stage_rows<VEC>(xs + (Ci + 1) * kPwLd, k.dy + q.b * Co * k.P, Co, k.P, q.p0, q.np);
    stage_rows<VEC>(xs + (Ci + 1 + Co) * kPwLd, k.gs + q.b * Co * k.P, Co, k.P, q.p0, q.np);
    cp_async_commit();
  };
  long long tile = blockIdx.x;
  if (tile < ntiles) issue(tile, 0);
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const int st = (k.nstage == 2) ? (it & 1) : 0;
    const long long nxt = tile + gridDim.x;
    if (k.nstage == 2 && nxt < ntiles) {
      issue(nxt, st ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // every thread's copies of this tile have landed
    const TileOf q = tile_of(tile, tpb, k.P);
    const int np = q.np;
    float* xs = stage + st * RS * kPwLd;
    float* ds = xs + (Ci + 1) * kPwLd;
    {
      const int t = tid;
      const bool in = t < np;
      xs[Ci * kPwLd + t] = in ? 1.f : 0.f;
      if (in) {  // dA for this thread's point, kept in the tile and written out
        const float* gr = ds + Co * kPwLd;
        float* dout = k.da + (q.b * Co) * k.P + q.p0 + t;
#pragma unroll 4
        for (int o = 0; o < Co; ++o) {
          const float v = ds[o * kPwLd + t] * gr[o * kPwLd + t];
          ds[o * kPwLd + t] = v;
          dout[(long long)o * k.P] = v;
        }
      }
    }
    __syncthreads();  // the ones row and dA are in place
    float acc[kDaMT][kDaNT][4];
#pragma unroll
    for (int m = 0; m < kDaMT; ++m)
#pragma unroll
      for (int n = 0; n < kDaNT; ++n)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[m][n][e] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const int k0 = 32 * warp + 8 * kk;
      if (k0 >= np) break;  // past the tile's end every operand is zero
      uint32_t ab[kDaMT][4], as[kDaMT][4];
#pragma unroll
      for (int m = 0; m < kDaMT; ++m) {
        if (m < MT) {
          tf32_split(xs[xr[m][0] + k0 + c], ab[m][0], as[m][0]);
          tf32_split(xs[xr[m][1] + k0 + c], ab[m][1], as[m][1]);
          tf32_split(xs[xr[m][0] + k0 + c + 4], ab[m][2], as[m][2]);
          tf32_split(xs[xr[m][1] + k0 + c + 4], ab[m][3], as[m][3]);
        }
      }
#pragma unroll
      for (int n = 0; n < kDaNT; ++n) {
        if (n < NT) {
          uint32_t bb0, bs0, bb1, bs1;
          tf32_split(ds[dr[n] + k0 + c], bb0, bs0);
          tf32_split(ds[dr[n] + k0 + c + 4], bb1, bs1);
#pragma unroll
          for (int m = 0; m < kDaMT; ++m) {
            if (m < MT) {
              mma_tf32(acc[m][n], as[m], bb0, bb1);
              mma_tf32(acc[m][n], ab[m], bs0, bs1);
              mma_tf32(acc[m][n], ab[m], bb0, bb1);
            }
          }
        }
      }
    }
#pragma unroll
    for (int m = 0; m < kDaMT; ++m)
#pragma unroll
      for (int n = 0; n < kDaNT; ++n)
#pragma unroll
        for (int e = 0; e < 4; ++e) {  // Kahan: sum - cmp tracks the exact total
          const float yv = acc[m][n][e] - cmp[m][n][e];
          const float tv = sum[m][n][e] + yv;
          cmp[m][n][e] = (tv - sum[m][n][e]) - yv;
          sum[m][n][e] = tv;
        }
    __syncthreads();  // stage st is free for the copies issued next
    if (k.nstage == 1 && nxt < ntiles) issue(nxt, 0);
  }
  // fold: fold[warp][pair], then a fixed-order sum over the warps per pair
  cp_async_wait<0>();
  __syncthreads();
#pragma unroll
  for (int m = 0; m < kDaMT; ++m)
#pragma unroll
    for (int n = 0; n < kDaNT; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = 16 * m + g + 8 * (e >> 1), o = 8 * n + 2 * c + (e & 1);
        if (m < MT && n < NT && i <= Ci && o < Co)
          fold[warp * npair + (i < Ci ? i * Co + o : Ci * Co + o)] = sum[m][n][e] - cmp[m][n][e];
      }
  __syncthreads();
  for (int e = tid; e < npair; e += kPwThreads) {
    float s = 0.f, cc = 0.f;
    for (int w = 0; w < kPwThreads / 32; ++w) {
      const float yv = fold[w * npair + e] - cc;
      const float tv = s + yv;
      cc = (tv - s) - yv;
      s = tv;
    }
    k.part[(long long)blockIdx.x * npair + e] = s;
  }
}

// ---------------------------------------------------------------------------
// loss
// ---------------------------------------------------------------------------
template <int V>
__global__ void __launch_bounds__(kPwThreads) k_mse(const float* __restrict__ y,
                                                    const float* __restrict__ t, float* dy,
                                                    long long n, float scale,
                                                    float* __restrict__ part) {
  __shared__ float red[kPwThreads];
  float s = 0.f, c = 0.f;
  const long long nv = n / V;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nv;
       e += (long long)gridDim.x * blockDim.x) {
    float r[V];
    if (V == 4) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(y) + e);
      const float4 b = __ldg(reinterpret_cast<const float4*>(t) + e);
      r[0] = a.x - b.x;
      r[V > 1 ? 1 : 0] = a.y - b.y;
      r[V > 2 ? 2 : 0] = a.z - b.z;
      r[V > 3 ? 3 : 0] = a.w - b.w;
      if (dy) {
        float4 g;
        g.x = r[0] * scale;
        g.y = r[V > 1 ? 1 : 0] * scale;
        g.z = r[V > 2 ? 2 : 0] * scale;
        g.w = r[V > 3 ? 3 : 0] * scale;
        reinterpret_cast<float4*>(dy)[e] = g;
      }
    } else {
      r[0] = __ldg(y + e) - __ldg(t + e);
      if (dy) dy[e] = r[0] * scale;
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const float yv = r[v] * r[v] - c;
      const float tv = s + yv;
      c = (tv - s) - yv;
      s = tv;
    }
  }
  red[threadIdx.x] = s - c;
  __syncthreads();
  for (int h = kPwThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kPwThreads) k_mse_final(const float* __restrict__ part,
                                                          int rows, long long n, float* loss) {
  __shared__ float red[kPwThreads];
  float s = 0.f, c = 0.f;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    const float yv = part[r] - c;
    const float tv = s + yv;
    c = (tv - s) - yv;
    s = tv;
  }
  red[threadIdx.x] = s - c;
  __syncthreads();
  for (int h = kPwThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / (float)n;
}

// ---------------------------------------------------------------------------
// training step: Adam (Kingma and Ba), in place, FP32 state
//   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2
//   p = p - lr (m / bc1) / (sqrt(v / bc2) + eps),  bc = 1 - beta^t
// Grid-stride, 16-byte vectors when every pointer allows; 28 bytes per element.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void adam1(float& p, float g, float& m, float& v, float lr, float b1,
                                      float b2, float eps, float rbc1, float rbc2) {
  m = fmaf(b1, m, (1.f - b1) * g);
  v = fmaf(b2, v, (1.f - b2) * g * g);
  p -= lr * (m * rbc1) / (sqrtf(v * rbc2) + eps);
}

template <int V>
__global__ void __launch_bounds__(kPwThreads) k_adam(float* __restrict__ p,
                                                     const float* __restrict__ g,
                                                     float* __restrict__ m, float* __restrict__ v,
                                                     long long n, float lr, float b1, float b2,
                                                     float eps, float rbc1, float rbc2) {
  const long long nv = n / V;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nv;
       e += (long long)gridDim.x * blockDim.x) {
    if (V == 4) {
      float4 pp = reinterpret_cast<float4*>(p)[e];
      const float4 gg = __ldg(reinterpret_cast<const float4*>(g) + e);
      float4 mm = reinterpret_cast<float4*>(m)[e];
      float4 vv = reinterpret_cast<float4*>(v)[e];
      adam1(pp.x, gg.x, mm.x, vv.x, lr, b1, b2, eps, rbc1, rbc2);
      adam1(pp.y, gg.y, mm.y, vv.y, lr, b1, b2, eps, rbc1, rbc2);
      adam1(pp.z, gg.z, mm.z, vv.z, lr, b1, b2, eps, rbc1, rbc2);
      adam1(pp.w, gg.w, mm.w, vv.w, lr, b1, b2, eps, rbc1, rbc2);
      reinterpret_cast<float4*>(p)[e] = pp;
      reinterpret_cast<float4*>(m)[e] = mm;
      reinterpret_cast<float4*>(v)[e] = vv;
    } else {
      adam1(p[e], __ldg(g + e), m[e], v[e], lr, b1, b2, eps, rbc1, rbc2);
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int pw_blocks_per_sm(const void* kern, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kPwThreads, smem) != cudaSuccess ||
      nb < 1)
    nb = 1;
  return nb;
}

template <bool VEC>
static const void* pw_bwd_kernel(int KB) {
  switch (KB) {
    case 1: return reinterpret_cast<const void*>(k_pw_bwd<1, VEC>);
    case 2: return reinterpret_cast<const void*>(k_pw_bwd<2, VEC>);
    default: return reinterpret_cast<const void*>(k_pw_bwd<4, VEC>);
  }
}

static void allow_smem(const void* kern, size_t smem) {
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

size_t pointwise_smem_bytes(int Ci, int Co, bool saved_grad) {
  return pw_plan(Ci, Co, saved_grad).smem;
}

// The backward's grid, and so the rows of partial sums its workspace holds: the
// smaller occupancy of its two copy variants, with the shared-memory limit
// raised before the query, so the workspace query and every launch agree.
int pointwise_max_grid(int Ci, int Co) {
  const PwPlan pl = pw_plan(Ci, Co);
  const void* kv = pw_bwd_kernel<true>(pl.KB);
  const void* ks = pw_bwd_kernel<false>(pl.KB);
  allow_smem(kv, pl.smem);
  allow_smem(ks, pl.smem);
  const int nb = std::min(pw_blocks_per_sm(kv, pl.smem), pw_blocks_per_sm(ks, pl.smem));
  return sm_count() * std::min(8, nb);
}

int pointwise_npair(int Ci, int Co) { return pw_plan(Ci, Co).npair; }

static bool rows_aligned(long long P, const void* a, const void* b) {
  return (P % 4 == 0) && ((uintptr_t)a % 16 == 0) && (!b || (uintptr_t)b % 16 == 0);
}

cudaError_t launch_pointwise_fwd(const float* x, const float* w, const float* bias, float* y,
                                 int64_t B, int64_t P, int Ci, int Co, int act, cudaStream_t s) {
  PwArgs a{};
  a.x = x;
  a.w = w;
  a.bias = bias;
  a.y = y;
  a.B = B;
  a.P = P;
  a.Ci = Ci;
  a.Co = Co;
  a.act = act;
  const size_t smem = sizeof(float) * ((size_t)Ci * Co + Co);
  const bool vec = rows_aligned(P, x, y);
  const int V = vec ? 4 : 1;
  const long long items = B * ((P + V - 1) / V);
  const void* kern = vec ? reinterpret_cast<const void*>(k_pw_fwd<4>)
                         : reinterpret_cast<const void*>(k_pw_fwd<1>);
  const long long cap = (long long)sm_count() * pw_blocks_per_sm(kern, smem);
  const int grid = (int)std::max<long long>(1, std::min<long long>(cap, (items + kPwThreads - 1) / kPwThreads));
  if (vec)
    FNO_LAUNCH("fno_pointwise_fwd", k_pw_fwd<4>, grid, kPwThreads, smem, s, a);
  else
    FNO_LAUNCH("fno_pointwise_fwd", k_pw_fwd<1>, grid, kPwThreads, smem, s, a);
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// The block's 1x1 linear, bias and GELU for grids that the fused epilogues do
// not tile, around the spectral part S synthesised into out:
//   forward  A = out + bias + sum_i W(i, c) x[i];  out = GELU(A), gp = GELU'(A)
//   dX       out = sum_i W(i, c) x[i]   (before S is added to out)
// W(i, c) = w[i w_si + c w_sc].  A thread owns one point and holds all of its
// outputs before it writes any, so x may be out itself (dA kept in dx).
// FP32 on the CUDA cores, like the other pointwise layers.
// ---------------------------------------------------------------------------
struct PwAdd {
  const float* x;
  const float* w;
  const float* bias;  // forward only (nullable)
  float* out;
  float* gp;          // forward, nullable
  long long B, P;
  int Cl, Cs, w_si, w_sc, fwd;
};

template <int CM>
__global__ void __launch_bounds__(kPwThreads, 2) k_pw_add(const PwAdd k) {
  extern __shared__ __align__(16) float sma[];
  float* ws = sma;               // [Cl][CM], zero past Cs
  float* bs = sma + k.Cl * CM;   // [CM]
  for (int e = threadIdx.x; e < k.Cl * CM; e += blockDim.x) {
    const int i = e / CM, c = e - i * CM;
    ws[e] = (c < k.Cs) ? k.w[(long long)i * k.w_si + (long long)c * k.w_sc] : 0.f;
  }
  for (int c = threadIdx.x; c < CM; c += blockDim.x) bs[c] = (k.fwd && k.bias && c < k.Cs) ? k.bias[c] : 0.f;
  __syncthreads();
  const long long items = k.B * k.P;
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const long long b = it / k.P, p = it - b * k.P;
    const float* xb = k.x + b * k.Cl * k.P + p;
    float* ob = k.out + b * k.Cs * k.P + p;
    // every load of the point first, so that they are all in flight at once
    // (plain loads: x may alias out)
    float acc[CM], xv[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) xv[i] = (i < k.Cl) ? xb[(long long)i * k.P] : 0.f;
#pragma unroll
    for (int c = 0; c < CM; ++c) acc[c] = bs[c] + ((k.fwd && c < k.Cs) ? ob[(long long)c * k.P] : 0.f);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      if (i >= k.Cl) break;
      const float4* wr = reinterpret_cast<const float4*>(ws + i * CM);
#pragma unroll
      for (int c4 = 0; c4 < CM / 4; ++c4) {
        const float4 wv = wr[c4];
        acc[4 * c4 + 0] = fmaf(xv[i], wv.x, acc[4 * c4 + 0]);
        acc[4 * c4 + 1] = fmaf(xv[i], wv.y, acc[4 * c4 + 1]);
        acc[4 * c4 + 2] = fmaf(xv[i], wv.z, acc[4 * c4 + 2]);
        acc[4 * c4 + 3] = fmaf(xv[i], wv.w, acc[4 * c4 + 3]);
      }
    }
    float* gb = k.gp ? k.gp + b * k.Cs * k.P + p : nullptr;
#pragma unroll
    for (int c = 0; c < CM; ++c) {
      if (c < k.Cs) {
        const float a = acc[c];
        if (k.fwd) {
          float phi2, e;
          phi2_as(a, phi2, e);
          ob[(long long)c * k.P] = 0.5f * a * phi2;  // gelu_as(a)
          if (gb) gb[(long long)c * k.P] = fmaf(a * e, 0.39894228040143268f, 0.5f * phi2);  // gelu_grad_as(a)
        } else {
          ob[(long long)c * k.P] = a;
        }
      }
    }
  }
}

bool pw_add_supported(int Cl, int Cs) { return Cl >= 1 && Cl <= 32 && Cs >= 1 && Cs <= 32; }

template <int CM>
static cudaError_t launch_pw_add_t(const PwAdd& a, cudaStream_t s) {
  const size_t smem = sizeof(float) * ((size_t)a.Cl * CM + CM);
  const long long items = a.B * a.P;
  const long long cap = (long long)sm_count() * pw_blocks_per_sm((const void*)k_pw_add<CM>, smem);
  const int grid = (int)std::max<long long>(1, std::min<long long>(cap, (items + kPwThreads - 1) / kPwThreads));
  FNO_LAUNCH(a.fwd ? "fno_pw_add_fwd" : "fno_pw_add_dx", k_pw_add<CM>, grid, kPwThreads, smem, s, a);
  return cudaSuccess;
}

cudaError_t launch_pw_add(const float* x, const float* w, int w_si, int w_sc, const float* bias, float* out,
                          float* gp, int64_t B, int64_t P, int Cl, int Cs, bool fwd, cudaStream_t s) {
  if (B <= 0 || P <= 0) return cudaSuccess;
  if (!pw_add_supported(Cl, Cs)) return cudaErrorInvalidValue;
  PwAdd a{};
  a.x = x;
  a.w = w;
  a.bias = bias;
  a.out = out;
  a.gp = gp;
  a.B = B;
  a.P = P;
  a.Cl = Cl;
  a.Cs = Cs;
  a.w_si = w_si;
  a.w_sc = w_sc;
  a.fwd = fwd ? 1 : 0;
  if (Cs <= 8) return launch_pw_add_t<8>(a, s);
  if (Cs <= 16) return launch_pw_add_t<16>(a, s);
  if (Cs <= 24) return launch_pw_add_t<24>(a, s);
  return launch_pw_add_t<32>(a, s);
}

cudaError_t launch_pointwise_bwd(const float* x, const float* w, const float* bias,
                                 const float* dy, float* dx, float* part, int64_t B, int64_t P,
                                 int Ci, int Co, int act, int* rows_out, cudaStream_t s) {
  const PwPlan pl = pw_plan(Ci, Co);
  PwArgs a{};
  a.x = x;
  a.w = w;
  a.bias = bias;
  a.dy = dy;
  a.dx = dx;
  a.part = part;
  a.B = B;
  a.P = P;
  a.Ci = Ci;
  a.Co = Co;
  a.act = act;
  a.nstage = pl.nstage;
  const size_t stage_floats =
      (std::max(pl.nstage * sizeof(float) * (size_t)(Ci + 1 + Co) * kPwLd,
                sizeof(float) * (size_t)pl.S * pl.npair) + sizeof(float) - 1) / sizeof(float);
  const long long ntiles = B * ((P + kPwTile - 1) / kPwTile);
  const int grid = (int)std::max<long long>(1, std::min<long long>(pointwise_max_grid(Ci, Co), ntiles));
  const bool vec = rows_aligned(P, x, dy);
#define PW_BWD(KB_, V_)                                                                       \
  FNO_LAUNCH("fno_pointwise_bwd", (k_pw_bwd<KB_, V_>), grid, kPwThreads, pl.smem, s, a, pl.nbo, \
             pl.nblk, pl.S, stage_floats)
  if (vec) {
    switch (pl.KB) {
      case 1: PW_BWD(1, true); break;
      case 2: PW_BWD(2, true); break;
      default: PW_BWD(4, true); break;
    }
  } else {
    switch (pl.KB) {
      case 1: PW_BWD(1, false); break;
      case 2: PW_BWD(2, false); break;
      default: PW_BWD(4, false); break;
    }
  }
#undef PW_BWD
  *rows_out = grid;
  return cudaSuccess;
}

// tensor-core form of the pass (k_da_mma): staged rows, stages (two when two
// CTAs per SM still fit), shared-memory bytes
bool pointwise_da_mma_fits(int Ci, int Co) { return Ci + 1 <= 16 * kDaMT && Co <= 8 * kDaNT; }
static void da_mma_plan(int Ci, int Co, int& nstage, size_t& smem) {
  const size_t stage = sizeof(float) * (size_t)(Ci + 1 + 2 * Co) * kPwLd;
  nstage = (2 * stage <= 110 * 1024) ? 2 : 1;
  smem = std::max(nstage * stage, sizeof(float) * (size_t)(kPwThreads / 32) * (Ci * Co + Co));
}

static cudaError_t launch_da_mma(const float* x, const float* g, const float* dz, float* da,
                                 float* part, int max_rows, int64_t B, int64_t P, int Ci, int Co,
                                 int* rows_out, cudaStream_t s) {
  int nstage;
  size_t smem;
  da_mma_plan(Ci, Co, nstage, smem);
  PwArgs a{};
  a.x = x;
  a.dy = dz;
  a.gs = g;
  a.da = da;
  a.part = part;
  a.B = B;
  a.P = P;
  a.Ci = Ci;
  a.Co = Co;
  a.nstage = nstage;
  const long long ntiles = B * ((P + kPwTile - 1) / kPwTile);
  const void* kv = reinterpret_cast<const void*>(k_da_mma<true>);
  const void* ks = reinterpret_cast<const void*>(k_da_mma<false>);
  allow_smem(kv, smem);
  allow_smem(ks, smem);
  const int nb = std::min(pw_blocks_per_sm(kv, smem), pw_blocks_per_sm(ks, smem));
  long long grid = (long long)sm_count() * std::min(8, nb);
  grid = std::min<long long>(grid, ntiles);
  grid = std::min<long long>(grid, max_rows);
  if (grid < 1) grid = 1;
  if (rows_aligned(P, x, dz) && rows_aligned(P, g, nullptr))
    FNO_LAUNCH("fno_da_saved", k_da_mma<true>, (int)grid, kPwThreads, smem, s, a);
  else
    FNO_LAUNCH("fno_da_saved", k_da_mma<false>, (int)grid, kPwThreads, smem, s, a);
  *rows_out = (int)grid;
  return cudaSuccess;
}

cudaError_t launch_pointwise_bwd_saved(const float* x, const float* g, const float* dz, float* da,
                                       float* part, int max_rows, int64_t B, int64_t P, int Ci,
                                       int Co, int* rows_out, cudaStream_t s) {
  if (pointwise_da_mma_fits(Ci, Co))
    return launch_da_mma(x, g, dz, da, part, max_rows, B, P, Ci, Co, rows_out, s);
  // wider layers: the FP32 pair-block contraction of k_pw_bwd
  const PwPlan pl = pw_plan(Ci, Co, true);
  PwArgs a{};
  a.x = x;
  a.dy = dz;
  a.gs = g;
  a.da = da;
  a.part = part;
  a.B = B;
  a.P = P;
  a.Ci = Ci;
  a.Co = Co;
  a.act = 0;
  a.nstage = pl.nstage;
  const size_t stage_floats =
      (std::max(pl.nstage * sizeof(float) * (size_t)(Ci + 1 + 2 * Co) * kPwLd,
                sizeof(float) * (size_t)pl.S * pl.npair) + sizeof(float) - 1) / sizeof(float);
  const long long ntiles = B * ((P + kPwTile - 1) / kPwTile);
  const void* kv = pw_bwd_kernel<true>(pl.KB);
  const void* ks = pw_bwd_kernel<false>(pl.KB);
  allow_smem(kv, pl.smem);
  allow_smem(ks, pl.smem);
  const int nb = std::min(pw_blocks_per_sm(kv, pl.smem), pw_blocks_per_sm(ks, pl.smem));
  long long grid = (long long)sm_count() * std::min(8, nb);
  grid = std::min<long long>(grid, ntiles);
  grid = std::min<long long>(grid, max_rows);
  if (grid < 1) grid = 1;
  const bool vec = rows_aligned(P, x, dz) && rows_aligned(P, g, da);
#define PW_BWD(KB_, V_)                                                                       \
  FNO_LAUNCH("fno_da_saved", (k_pw_bwd<KB_, V_>), (int)grid, kPwThreads, pl.smem, s, a, pl.nbo, \
             pl.nblk, pl.S, stage_floats)
  if (vec) {
    switch (pl.KB) {
      case 1: PW_BWD(1, true); break;
      case 2: PW_BWD(2, true); break;
      default: PW_BWD(4, true); break;
    }
  } else {
    switch (pl.KB) {
      case 1: PW_BWD(1, false); break;
      case 2: PW_BWD(2, false); break;
      default: PW_BWD(4, false); break;
    }
  }
#undef PW_BWD
  *rows_out = (int)grid;
  return cudaSuccess;
}

int mse_max_grid() { return sm_count() * 4; }

cudaError_t launch_mse(const float* y, const float* t, float* dy, int64_t n, float* loss,
                       float* part, cudaStream_t s) {
  const bool vec = (n % 4 == 0) && ((uintptr_t)y % 16 == 0) && ((uintptr_t)t % 16 == 0) &&
                   (!dy || (uintptr_t)dy % 16 == 0);
  const long long nv = vec ? n / 4 : n;
  const int grid = (int)std::max<long long>(1, std::min<long long>(mse_max_grid(), (nv + kPwThreads - 1) / kPwThreads));
  const float scale = (float)(2.0 / (double)n);
  if (vec)
    FNO_LAUNCH("fno_mse", k_mse<4>, grid, kPwThreads, 0, s, y, t, dy, (long long)n, scale, part);
  else
    FNO_LAUNCH("fno_mse", k_mse<1>, grid, kPwThreads, 0, s, y, t, dy, (long long)n, scale, part);
  FNO_LAUNCH("fno_mse_final", k_mse_final, 1, kPwThreads, 0, s, part, grid, (long long)n, loss);
  return cudaSuccess;
}

}  // namespace fno

namespace fno {

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr,
                        float b1, float b2, float eps, double bc1, double bc2, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const bool vec = (n % 4 == 0) && ((uintptr_t)p % 16 == 0) && ((uintptr_t)g % 16 == 0) &&
                   ((uintptr_t)m % 16 == 0) && ((uintptr_t)v % 16 == 0);
  const long long nv = vec ? n / 4 : n;
  const int grid = (int)std::max<long long>(
      1, std::min<long long>((long long)sm_count() * 8, (nv + kPwThreads - 1) / kPwThreads));
  const float rbc1 = (float)(1.0 / bc1), rbc2 = (float)(1.0 / bc2);
  if (vec)
    FNO_LAUNCH("fno_adam", k_adam<4>, grid, kPwThreads, 0, s, p, g, m, v, (long long)n, lr, b1, b2,
               eps, rbc1, rbc2);
  else
    FNO_LAUNCH("fno_adam", k_adam<1>, grid, kPwThreads, 0, s, p, g, m, v, (long long)n, lr, b1, b2,
               eps, rbc1, rbc2);
  return cudaSuccess;
}

}  // namespace fno
