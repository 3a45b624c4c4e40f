// fno_internal.h -- declarations shared by the translation units of libfno.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fno.h"

namespace fno {

// Sizes with the derived mode counts.  Jx = 2mx, Jy = 2my, Jz = 2mz, Jt = mt;
// Ng = grid points per channel, Mk = kept modes per channel.
struct Dims {
  int64_t B, Ci, Co, Nx, Ny, Nz, Nt, mx, my, mz, mt;
  int64_t Jx, Jy, Jz, Jt, Ng, Mk;
};

// DFT basis tables in the workspace, FP32 complex (re, im), generated in FP64.
//   forward  F?[j][n] = exp(-2 pi i k_j n / N?)          (Fx, Fy, Fz, Ft)
//            Fta[j][t] = (c(kt)/N) exp(-2 pi i kt t / Nt)   (the adjoint scale of G)
//   inverse  I?[n][j] = exp(+2 pi i k_j n / N?)          (Ix, Iy, Iz)
//            Its[j][t] = (c(kt)/N) exp(+2 pi i kt t / Nt)   (the block's inverse)
//            Itu[j][t] = exp(+2 pi i kt t / Nt)             (adjoint of the forward DFT)
struct Tables {
  float2 *Fx, *Fy, *Fz, *Ft, *Fta;
  float2 *Ix, *Iy, *Iz, *Its, *Itu;
};

// ---- launch bookkeeping (fno_api.cu) --------------------------------------
void prof_before(const char* name, cudaStream_t s);
void prof_after(cudaStream_t s);
int sm_count();

// ---- FP32 CUDA-core kernels (fno_fp32.cu) -----------------------------------
// also clears the device status word *err of the call
cudaError_t launch_tables(const Dims& d, const Tables& T, int* err, cudaStream_t s);

// in[ncol][Nz][Nt] real -> out[ncol][Jz][Jt] complex: pruned DFT over t, then z.
// ft is Ft or Fta.
cudaError_t launch_fwd_tz_f32(const float* in, float2* out, int64_t ncol, const Dims& d,
                              const float2* ft, const float2* fz, cudaStream_t s);

// out[o][q][i] = sum_n tab[q][n] in[o][n][i] (complex), tab [nout][nin].
cudaError_t launch_line_f32(const float2* in, float2* out, int64_t outer, int nin, int nout,
                            int64_t inner, const float2* tab, cudaStream_t s);

// yh[b][o][j] = sum_i xh[b][i][j] w[i][o][j]
cudaError_t launch_mix_f32(const Dims& d, const float2* xh, const float2* w, float2* yh,
                           cudaStream_t s);

// dw[i][o][j] = sum_b conj(xh[b][i][j]) g[b][o][j] (nullable),
// gxh[b][i][j] = sum_o conj(w[i][o][j]) g[b][o][j] (nullable)
cudaError_t launch_mix_adjoint_f32(const Dims& d, const float2* xh, const float2* w,
                                   const float2* g, float2* dw, float2* gxh, cudaStream_t s);

enum EpiMode { EPI_SPECTRAL = 0, EPI_FWD = 1, EPI_DA = 2, EPI_DX = 3 };

struct EpiArgs {
  int mode;
  const float2* U;      // [B][Cs][Nx][Ny][Jz][Jt]   spectrum after the inverse x, y stages
  const float* lin_in;  // [B][Cl][grid]  x (FWD, DA) or dA (DX)
  const float* wlin;    // [Ci][Co]
  const float* bias;    // [Co]
  const float* dz;      // [B][Co][grid] (DA)
  float* out;           // [B][Cs][grid]
  float* gp;            // FWD, nullable: GELU'(A) [B][Cs][grid] for a training forward
  float* part;          // per-CTA partial sums of dWl and db (DA)
  const float2* Iz;     // [Nz][Jz]
  const float2* It;     // [Jt][Nt]  (Its or Itu)
  int Cs, Cl;           // output (spectral) channels, linear-input channels
  int w_si, w_sc;       // w_lin index of (linear-input channel i, output channel c) = i*w_si + c*w_sc
};

// Inverse z, t stages with the pointwise epilogue; returns the grid size used
// (the number of partial rows written in EPI_DA mode).
cudaError_t launch_epilogue_f32(const Dims& d, const EpiArgs& a, int* grid_used, cudaStream_t s);
int epilogue_max_grid();
size_t epilogue_smem_bytes(const Dims& d, int mode, int Cs, int Cl);
size_t fwd_tz_smem_bytes(const Dims& d);
size_t line_smem_bytes(int nin, int nout);

// dwl[i][o] = sum_r part[r][i*Co+o], db[o] = sum_r part[r][Ci*Co+o]
cudaError_t launch_reduce_partials(const float* part, int rows, int Ci, int Co, float* dwl,
                                   float* db, cudaStream_t s);

cudaError_t launch_fill_zero(float* p, int64_t n, cudaStream_t s);

// Inverse z, t + epilogue on warp-level mma.sync (fno_mma.cu), BF16 or split
// BF16; same contract as launch_epilogue_f32.  table: device scratch of
// epilogue_mma_table_bytes(d) for the basis fragments.
bool epilogue_mma_supported(const Dims& d, int mode, int Cs, int Cl, char* why, size_t nwhy);
size_t epilogue_mma_table_bytes(const Dims& d);
cudaError_t launch_epilogue_mma(const Dims& d, const EpiArgs& a, bool split, bool tf32, void* table,
                                int* err, int* grid_used, cudaStream_t s);

// Inverse z, t + epilogue on the 5th-generation tensor cores (fno_tc.cu):
// tcgen05.mma into TMEM accumulators, modes EPI_FWD, EPI_DX and EPI_SPECTRAL;
// same contract as launch_epilogue_f32 (no partial sums).  table: device
// scratch of epilogue_tc_table_bytes(d) for the z basis images.
bool epilogue_tc_supported(const Dims& d, int mode, int Cs, int Cl, char* why, size_t nwhy);
size_t epilogue_tc_table_bytes(const Dims& d);
cudaError_t launch_epilogue_tc(const Dims& d, const EpiArgs& a, bool split, bool tf32, void* table, int* err,
                               cudaStream_t s);

// One complex DFT axis on mma.sync (fno_mma.cu), BF16 (one product), split
// BF16 (three-way splits, six products) or TF32 (operands rounded to TF32, then
// split); same contract as launch_line_f32.
bool line_mma_supported(int nin, int nout);
cudaError_t launch_line_mma(const float2* in, float2* out, int64_t outer, int nin, int nout,
                            int64_t inner, const float2* tab, bool split, bool tf32, cudaStream_t s);
// The inverse t stage to real points on mma.sync (fno_mma.cu), for grids the
// fused epilogues do not tile: out[r][t] (+)= sum_jt Re(It[jt][t] V[r][jt]),
// r < R, t < Nt <= 128, Jt <= 8; accumulate adds to out instead of writing it.
// Precisions as launch_line_mma.
bool synth_t_supported(int Nt, int Jt);
cudaError_t launch_synth_t(const float2* V, float* out, int64_t R, int Nt, int Jt, const float2* It,
                           bool accumulate, bool split, bool tf32, cudaStream_t s);

// ---- layers around the blocks (fno_pointwise.cu) ---------------------------
// y[b,o,p] = act(sum_i x[b,i,p] w[i,o] + bias[o]) (bias nullable, act 0/1 = none/GELU).
cudaError_t launch_pointwise_fwd(const float* x, const float* w, const float* bias, float* y,
                                 int64_t B, int64_t P, int Ci, int Co, int act, cudaStream_t s);
// dA = dy act'(A); dx = W dA (nullable); writes rows_out rows of per-CTA partial
// sums [row][Ci*Co + Co] of (dw, db) into part, for launch_reduce_partials.
cudaError_t launch_pointwise_bwd(const float* x, const float* w, const float* bias,
                                 const float* dy, float* dx, float* part, int64_t B, int64_t P,
                                 int Ci, int Co, int act, int* rows_out, cudaStream_t s);
size_t pointwise_smem_bytes(int Ci, int Co, bool saved_grad = false);
// The block's 1x1 + bias + GELU in place around a synthesised spectral part
// (grids the fused epilogues do not tile): fwd out = GELU(out + bias + W x),
// gp = GELU'(same) (nullable); else out = W x (x may be out).  W(i, c) =
// w[i w_si + c w_sc]; Cl, Cs <= 32.
bool pw_add_supported(int Cl, int Cs);
cudaError_t launch_pw_add(const float* x, const float* w, int w_si, int w_sc, const float* bias, float* out,
                          float* gp, int64_t B, int64_t P, int Cl, int Cs, bool fwd, cudaStream_t s);
int pointwise_max_grid(int Ci, int Co);  // the most rows launch_pointwise_bwd writes
// The dA step of a block backward after a training forward: dA = dz * g (g the
// forward's GELU'(A)), written to da, with the (dW_lin, db) partial sums of
// x and dA; at most max_rows partial rows (the CTAs launched, *rows_out).
// the dA pass contracts dW_lin on the tensor cores (else on the CUDA cores)
bool pointwise_da_mma_fits(int Ci, int Co);
cudaError_t launch_pointwise_bwd_saved(const float* x, const float* g, const float* dz, float* da,
                                       float* part, int max_rows, int64_t B, int64_t P, int Ci,
                                       int Co, int* rows_out, cudaStream_t s);
// loss = mean((y - t)^2) into *loss, dy = 2 (y - t) / n (nullable); part: mse_max_grid() floats
int mse_max_grid();
cudaError_t launch_mse(const float* y, const float* t, float* dy, int64_t n, float* loss,
                       float* part, cudaStream_t s);
// Adam update in place; bc1, bc2 = 1 - beta1^t, 1 - beta2^t
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr,
                        float b1, float b2, float eps, double bc1, double bc2, cudaStream_t s);

// Pruned DFT over t then z with both stages on mma.sync (fno_mma.cu); same
// contract as launch_fwd_tz_f32.  err: device word set to nonzero when a
// bounded wait gives up.
bool fwd_tz_mma_supported(const Dims& d, char* why, size_t nwhy);
cudaError_t launch_fwd_tz_mma(const float* in, float2* out, int64_t ncol, const Dims& d,
                              const float2* ft, const float2* fz, bool split, bool tf32, int* err,
                              cudaStream_t s);

// The dA pass of a block backward after a training forward fused with the
// forward pruned t, z DFT of dA (fno_da_tz.cu, mma.sync): writes da, the
// spectrum t1 = [B Co Nx Ny][Jz][Jt] (ft = Fta) and at most max_rows partial
// rows of (dW_lin, db) (*rows_out, as launch_pointwise_bwd_saved).  err: device
// word set to nonzero when a bounded wait gives up.
bool da_tz_supported(const Dims& d, char* why, size_t nwhy);
cudaError_t launch_da_tz(const float* x, const float* g, const float* dz, float* da, float2* t1, float* part,
                         int max_rows, const Dims& d, const float2* ft, const float2* fz, bool split, bool tf32,
                         int* err, int* rows_out, cudaStream_t s);

#ifdef __CUDACC__
// Launch with the profiling hooks; returns the launch error from the caller.
#define FNO_LAUNCH(name, kern, grid, block, smem, stream, ...)   \
  do {                                                           \
    prof_before(name, stream);                                   \
    kern<<<grid, block, smem, stream>>>(__VA_ARGS__);            \
    cudaError_t e_ = cudaGetLastError();                         \
    prof_after(stream);                                          \
    if (e_ != cudaSuccess) return e_;                            \
  } while (0)
__device__ __forceinline__ float gelu_f(float a) {
  return 0.5f * a * (1.0f + erff(a * 0.70710678118654752440f));
}
__device__ __forceinline__ float gelu_grad_f(float a) {
  return 0.5f * (1.0f + erff(a * 0.70710678118654752440f)) +
         a * expf(-0.5f * a * a) * 0.39894228040143267794f;
}

// Phi2(a) = 1 + erf(a / sqrt 2) and exp(-a^2 / 2), with erf from Abramowitz
// and Stegun 7.1.26: erf(u) = 1 - (a1 t + ... + a5 t^5) exp(-u^2),
// t = 1 / (1 + p u), u >= 0, |error| < 1.5e-7.  For a < 0 the complement is
// taken directly (no cancellation).
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ void phi2_as(float a, float& phi2, float& e) {
  const float u = fabsf(a) * 0.70710678118654752f;
  const float t = rcp_approx(fmaf(0.3275911f, u, 1.0f));
  float q = fmaf(1.061405429f, t, -1.453152027f);
  q = fmaf(q, t, 1.421413741f);
  q = fmaf(q, t, -0.284496736f);
  q = fmaf(q, t, 0.254829592f);
  q *= t;
  e = ex2_approx(-u * u * 1.4426950408889634f);
  const float c = q * e;  // 1 - erf(u)
  phi2 = (a >= 0.f) ? 2.0f - c : c;
}
__device__ __forceinline__ float gelu_as(float a) {
  float phi2, e;
  phi2_as(a, phi2, e);
  return 0.5f * a * phi2;
}
__device__ __forceinline__ float gelu_grad_as(float a) {
  float phi2, e;
  phi2_as(a, phi2, e);
  return fmaf(a * e, 0.39894228040143268f, 0.5f * phi2);
}
#endif

}  // namespace fno
