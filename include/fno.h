/*
 * fno.h -- C ABI of the GB300 (sm_103a) spectral FNO block library (libfno.so).
 *
 * The block is the FNO block of the paper's Alg. 2 (Sec. IV-C): a truncated
 * real DFT of every channel onto the kept low modes (F then S), a complex
 * per-mode channel mixing with learned weights (the einsum of Alg. 2), the
 * zero-padded inverse DFT (S^T then F^T), and -- for the full block -- the
 * pointwise 1x1 channel linear with bias of the original FNO that Sec. IV-C
 * says the architecture follows, and the nonlinearity sigma of Alg. 1 (GELU,
 * exact erf form):
 *
 *   theta_j(p) = 2 pi (kx x/Nx + ky y/Ny + kz z/Nz + kt t/Nt)
 *   Xh[b,i,j]  = sum_p x[b,i,p] exp(-i theta_j(p))
 *   Yh[b,o,j]  = sum_i Xh[b,i,j] w[i,o,j]
 *   S[b,o,p]   = (1/N) sum_j c(kt_j) Re(Yh[b,o,j] exp(+i theta_j(p)))
 *   spectral:  y = S
 *   block:     z = GELU(S + sum_i x[b,i,p] w_lin[i,o] + bias[o])
 *
 * N = Nx Ny Nz Nt.  Kept modes: stored index jx < mx is frequency jx, jx >= mx
 * is jx - 2 mx (same for y, z); t keeps kt = 0..mt-1 (real half spectrum).
 * c(kt) = 1 at kt = 0 and at kt = Nt/2 (Nt even), 2 otherwise.
 *
 * Layouts (all C-contiguous, FP32, device memory):
 *   x, dx            [B][C_in ][Nx][Ny][Nz][Nt]
 *   y, z, dy, dz     [B][C_out][Nx][Ny][Nz][Nt]
 *   w, dw            [C_in][C_out][2mx][2my][2mz][mt][2]   (re, im interleaved)
 *   w_lin, dw_lin    [C_in][C_out]
 *   bias, db         [C_out]
 *
 * Ownership: the caller owns every buffer, including the workspace whose size
 * fno_workspace_bytes() returns; the library allocates no device memory.  The
 * DFT basis tables are regenerated into the workspace (FP64 arithmetic on the
 * device, stored in the precision the kernels read) on every call.
 *
 * Semantics: every call is asynchronous on the given stream (a cudaStream_t
 * passed as void*, NULL = legacy default stream).  Gradients overwrite their
 * outputs.  Inputs must not alias outputs.
 *
 * Errors: functions return an fno_status; nothing aborts or traps.  On any
 * error other than FNO_ERR_CUDA nothing has been enqueued.  fno_last_error()
 * returns a message for the calling thread's last failure.
 */
#ifndef FNO_GB300_FNO_H_
#define FNO_GB300_FNO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Problem sizes.  B >= 0 (B = 0 is an empty batch); every other entry >= 1,
 * 2 mx <= Nx, 2 my <= Ny, 2 mz <= Nz, mt <= Nt/2 + 1 (FNO_ERR_INVALID_ARG
 * otherwise).  Supported: C_in, C_out <= 64 and mt <= 16 (FNO_ERR_UNSUPPORTED
 * otherwise). */
typedef struct fno_dims {
  int64_t B, C_in, C_out, Nx, Ny, Nz, Nt, mx, my, mz, mt;
} fno_dims;

/* Arithmetic of the contractions (accumulation is always FP32):
 *   FNO_FP32    FP32 on the CUDA cores (the plain form)
 *   FNO_TF32    TF32 numerics: every tensor-core operand rounded to TF32
 *               (nearest), exact products; a TF32 value is exact as BF16
 *               hi + lo, so it runs as split products on the BF16 tensor
 *               cores (the cost of FNO_BF16X3, the accuracy of TF32)
 *   FNO_BF16    BF16 tensor-core products (one product)
 *   FNO_BF16X3  split BF16 on the tensor cores: hi + lo with three products
 *               in the DFT stages, three-way splits with six products in the
 *               line stages and the mma.sync 1x1 stages; the 1x1 of the fused
 *               tcgen05 epilogue as 3xTF32 (big + small parts, three
 *               products), FP32-like
 * The tensor-core precisions need Nt even and at most 128, Nz * Nt a multiple
 * of 4, mt <= 8 and 2 mz <= 64 (FNO_ERR_UNSUPPORTED otherwise).  The fused
 * inverse z, t + epilogue stage runs, in FNO_BF16X3 and FNO_TF32, on tcgen05
 * (TMEM accumulators) for Nt = 16 or 32, Nz a multiple of 512 / Nt, 2 mz <= 24
 * and up to 32 channels; on warp-level mma.sync for FNO_BF16, the other shapes
 * its tiling takes and the dA pass of fno_block_bwd.  Other Nt (the paper's 84
 * and 86), with mt <= 8, up to 32 channels and the inverse z stage within the
 * tensor-core line tiling, take a synthesis path: the inverse z stage and the
 * inverse t stage to real points on mma.sync, the second written straight into
 * the output, then the 1x1, bias and GELU in FP32 in place (a workspace region
 * of B * max(C_in, C_out) * Nx * Ny * Nz * mt complex values holds the z stage;
 * the recomputing backward's dA pass stays on the FP32 kernel).  The FP32
 * kernels run the rest. */
typedef enum fno_precision {
  FNO_FP32 = 0,
  FNO_TF32 = 1,
  FNO_BF16 = 2,
  FNO_BF16X3 = 3
} fno_precision;

typedef enum fno_status {
  FNO_OK = 0,
  FNO_ERR_INVALID_ARG = -1, /* null required pointer, bad size, bad precision or op */
  FNO_ERR_UNSUPPORTED = -2, /* valid sizes the kernels do not handle (message says which) */
  FNO_ERR_WORKSPACE = -3,   /* workspace too small or misaligned (256-byte alignment) */
  FNO_ERR_CUDA = -4,        /* a CUDA call failed; message carries its error string */
  FNO_ERR_TIMEOUT = -5      /* a bounded device-side wait gave up */
} fno_status;

typedef enum fno_op {
  FNO_OP_SPECTRAL_FWD = 0,
  FNO_OP_SPECTRAL_BWD = 1,
  FNO_OP_BLOCK_FWD = 2,
  FNO_OP_BLOCK_BWD = 3,
  /* one workspace for fno_block_fwd_train and the fno_block_bwd_saved after
   * it: the FNO_OP_BLOCK_BWD layout plus GELU'(A), B * C_out * N floats */
  FNO_OP_BLOCK_TRAIN = 4
} fno_op;

/* Workspace bytes that op needs for these sizes and precision (0 on invalid
 * arguments; see fno_last_error()). */
size_t fno_workspace_bytes(const fno_dims* dims, int precision, int op);

/* Spectral convolution forward, y = S(x; w)  (Alg. 2: F, S, einsum, S^T, F^T).
 * x: input, w: complex weights, y: output; ws: workspace of ws_bytes. */
int fno_spectral_fwd(const fno_dims* dims, int precision, const float* x, const float* w,
                     float* y, void* ws, size_t ws_bytes, void* stream);

/* Spectral convolution backward for upstream gradient dy (Alg. 2 differentiated;
 * the inverse is the adjoint of the forward operators, Sec. IV-C):
 *   G   = (c(kt)/N) DFT(dy)
 *   dw  = sum_b conj(Xh) G          (dL/dRe w, dL/dIm w), nullable
 *   dx  = sum_j Re(sum_o conj(w) G exp(+i theta))   nullable
 * At least one of dx, dw must be non-null. */
int fno_spectral_bwd(const fno_dims* dims, int precision, const float* x, const float* w,
                     const float* dy, float* dx, float* dw, void* ws, size_t ws_bytes,
                     void* stream);

/* Full FNO block forward: z = GELU(S(x; w) + w_lin^T x + bias). */
int fno_block_fwd(const fno_dims* dims, int precision, const float* x, const float* w,
                  const float* w_lin, const float* bias, float* z, void* ws, size_t ws_bytes,
                  void* stream);

/* Block forward of a training step: computes z exactly as fno_block_fwd does
 * and also keeps GELU'(A) at every point in the workspace (B * C_out * N
 * floats), so that the fno_block_bwd_saved call after it forms dA = dz
 * GELU'(A) pointwise instead of evaluating the inverse transform and the 1x1
 * again (the derivative is the one of the erf form of GELU, Sec. IV-C's
 * block, taken at the forward's own A).  In the tensor-core precisions with
 * more than 31 input or 24 output channels (up to 32) re-evaluating A on the
 * tensor cores is the faster form: there the call skips the store and the
 * saved backward re-evaluates A, as after fno_block_fwd.  ws_bytes must cover
 * fno_workspace_bytes(dims, precision, FNO_OP_BLOCK_TRAIN) in every case; the
 * workspace is owned by the caller and must stay untouched until the
 * backward. */
int fno_block_fwd_train(const fno_dims* dims, int precision, const float* x, const float* w,
                        const float* w_lin, const float* bias, float* z, void* ws,
                        size_t ws_bytes, void* stream);

/* Full FNO block backward for upstream gradient dz.  The forward is recomputed
 * from x (activation checkpointing: only the block input is kept between the
 * passes).  dA = dz GELU'(A); db = sum dA; dw_lin = sum x dA^T; dw as in
 * fno_spectral_bwd with G = (c(kt)/N) DFT(dA); dx = S^T-path + w_lin dA.
 * All five outputs are required. */
int fno_block_bwd(const fno_dims* dims, int precision, const float* x, const float* w,
                  const float* w_lin, const float* bias, const float* dz, float* dx, float* dw,
                  float* dw_lin, float* db, void* ws, size_t ws_bytes, void* stream);

/* Block backward that reuses the forward's spectra instead of recomputing them.
 * After fno_block_fwd the workspace holds the input's kept spectrum Xh and the
 * inverse x, y partial of the output spectrum (together about 0.35 GB at width
 * 20 on 128^3 x 32, against 5.4 GB for the input); this call takes them from
 * there and runs only the adjoint chain, computing what fno_block_bwd
 * computes.  After fno_block_fwd_train it also takes GELU'(A) from there:
 * dA, dw_lin and db then come from one pointwise pass over x, dz and GELU'(A)
 * (FP32-accurate products, Kahan-summed), and agree with fno_block_bwd to
 * rounding rather than bitwise.  In the tensor-core precisions, for Nt = 16 or
 * 32, Nz a multiple of 16, mt <= 8, 2 mz <= 32, C_in <= 31 and C_out <= 24,
 * that pass also forms the t, z DFT of dA (the first stages of the dw and dx
 * spectra), so dA is written once and not read back for them.
 * Contract: ws (and ws_bytes, sized for FNO_OP_BLOCK_BWD after fno_block_fwd,
 * FNO_OP_BLOCK_TRAIN after fno_block_fwd_train) is the workspace of the last
 * forward call made with it, with the same dims, precision, x and w, and no
 * other call has used ws since; x and w are unchanged.  The library records
 * which forward call left its state in each workspace (host bookkeeping only)
 * and refuses with FNO_ERR_INVALID_ARG when the record does not match; it
 * cannot see writes to x or w made by the caller. */
int fno_block_bwd_saved(const fno_dims* dims, int precision, const float* x, const float* w,
                        const float* w_lin, const float* bias, const float* dz, float* dx,
                        float* dw, float* dw_lin, float* db, void* ws, size_t ws_bytes,
                        void* stream);

/* Status a previous call left in its workspace: waits for `stream`, then returns
 * FNO_OK, FNO_ERR_TIMEOUT when one of that call's bounded device-side waits
 * (tensor-core pipeline barriers) gave up and the kernel returned early, or
 * FNO_ERR_CUDA when a kernel found its shared-memory window misaligned for the
 * tensor copies and returned without computing. */
int fno_workspace_status(const void* ws, void* stream);

/* Message of the calling thread's last error ("" if none). */
const char* fno_last_error(void);

/* fno_status of the calling thread's last failure (FNO_OK if none), e.g. to tell
 * why fno_workspace_bytes() returned 0. */
int fno_last_status(void);

/* Library ABI version (major * 100 + minor). */
int fno_version(void);

/* Number of kernels this library has launched since it was loaded. */
int64_t fno_launch_count(void);

/* Optional per-kernel timing: while enabled, every launch is bracketed by CUDA
 * events on its own stream.  fno_profile_stop() waits for the recorded events
 * and aggregates them; fno_profile_entry() then reads kernel i's name, launch
 * count and summed device time.  Host-side bookkeeping only; not thread safe. */
int fno_profile_start(void);
int fno_profile_stop(void);
int fno_profile_count(void);
int fno_profile_entry(int i, const char** name, int64_t* launches, double* total_ms);

/* ---- layers around the blocks (Alg. 1) --------------------------------------
 * Alg. 1 wraps the FNO blocks in an encoder, a 1x1 convolution that lifts the
 * input channels to the width, and a decoder, a 1x1 convolution that brings the
 * width down to the output channels; each is followed by sigma.  The
 * pointwise layer is that 1x1 convolution over P points per channel (P = Nx Ny
 * Nz Nt on the 4-D grid), with an optional bias (the original FNO's 1x1 layers
 * carry one):
 *
 *   y[b,o,p] = act( sum_i x[b,i,p] w[i,o] + bias[o] )    act: FNO_ACT_NONE or
 *                                                        FNO_ACT_GELU (erf form)
 * Layouts (C-contiguous FP32, device memory): x, dx [B][C_in][P]; y, dy
 * [B][C_out][P]; w, dw [C_in][C_out]; bias, db [C_out].  1 <= C_in, C_out <= 64,
 * B >= 0, P >= 0 (an empty input gives zero dw, db).  FP32 on the CUDA cores in
 * every precision: with so few channels these layers are bound by HBM. */
typedef struct fno_pw_dims {
  int64_t B, C_in, C_out, P;
} fno_pw_dims;

typedef enum fno_act { FNO_ACT_NONE = 0, FNO_ACT_GELU = 1 } fno_act;

/* Forward.  bias nullable (zero).  No workspace. */
int fno_pointwise_fwd(const fno_pw_dims* dims, int act, const float* x, const float* w,
                      const float* bias, float* y, void* stream);

/* Workspace bytes of fno_pointwise_bwd for these sizes on the current device
 * (0 on invalid arguments). */
size_t fno_pointwise_workspace_bytes(const fno_pw_dims* dims);

/* Backward for upstream gradient dy: dA = dy act'(A) (A recomputed from x);
 * dx = w dA (nullable: the encoder's input needs none); dw = sum x dA^T and
 * db = sum dA over batch and points (db nullable), reduced in a fixed order. */
int fno_pointwise_bwd(const fno_pw_dims* dims, int act, const float* x, const float* w,
                      const float* bias, const float* dy, float* dx, float* dw, float* db,
                      void* ws, size_t ws_bytes, void* stream);

/* Workspace bytes of fno_mse_loss on the current device. */
size_t fno_mse_workspace_bytes(int64_t n);

/* Mean-squared-error training loss over n >= 1 values: *loss = (1/n) sum
 * (y - target)^2 (one device float), dy = (2/n)(y - target) (nullable), the sum
 * reduced in a fixed order. */
int fno_mse_loss(int64_t n, const float* y, const float* target, float* loss, float* dy,
                 void* ws, size_t ws_bytes, void* stream);

/* ---- training step -------------------------------------------------------------
 * One Adam update (Kingma and Ba; the optimizer of the original FNO -- the paper
 * does not name its own) of n parameters in place, FP32 state, step t >= 1:
 *   m = beta1 m + (1 - beta1) g;   v = beta2 v + (1 - beta2) g^2
 *   param -= lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps)
 * param, m, v read and written, grad read; all device pointers, 4-byte
 * aligned; m and v start at zero before step 1.  0 <= beta < 1, eps > 0,
 * lr >= 0.  Asynchronous on stream; no workspace. */
int fno_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr,
                  float beta1, float beta2, float eps, int64_t step, void* stream);

/* ---- allocation-free variant ------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot hand the library a workspace: for example a host program whose own
 * pool has reserved all device memory up front, or a runtime that forbids any
 * device allocation once it has started, so neither it nor its plug-ins may call
 * cudaMalloc to size a workspace.
 *
 * fno_spectral_fwd_static computes exactly what fno_spectral_fwd computes, but
 * takes its scratch from a fixed array in the library's device memory
 * (FNO_STATIC_SCRATCH_BYTES = 16 MiB, held on every GPU that loads the library
 * until the process exits) instead of a caller workspace.  The caller still
 * passes the input x, the weights w and the output y.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   - Sizes whose fno_workspace_bytes(dims, precision, FNO_OP_SPECTRAL_FWD)
 *     exceeds FNO_STATIC_SCRATCH_BYTES are refused with FNO_ERR_UNSUPPORTED
 *     before anything is enqueued.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before capturing any stream.  The lookup also loads the library's device
 *     code on that device, which is when the array's memory is committed: a
 *     host that reserves the rest of device memory up front calls
 *     fno_static_prepare() first.
 *   - The address is cached per device for the life of the process; it does
 *     not survive cudaDeviceReset, so these calls must not be used across one.
 *   - All calls share the one array and it keeps the previous call's contents;
 *     every byte a call reads from it is written earlier in the same call, so
 *     nothing needs clearing.  Calls that overlap on the GPU (other streams,
 *     other host threads) race on the array: serialise them.
 */
#define FNO_STATIC_SCRATCH_BYTES ((size_t)16 << 20)
int fno_spectral_fwd_static(const fno_dims* dims, int precision, const float* x, const float* w,
                            float* y, void* stream);

/* Looks up the static scratch on the current device, loading the library's
 * device code there (so committing the array's FNO_STATIC_SCRATCH_BYTES now
 * rather than at the first fno_spectral_fwd_static).  No allocation call is
 * made.  Returns FNO_OK or FNO_ERR_CUDA. */
int fno_static_prepare(void);

/* Status the last fno_spectral_fwd_static call on the current device left in
 * the static scratch: waits for `stream`, then returns FNO_OK,
 * FNO_ERR_TIMEOUT when one of that call's bounded device-side waits gave up,
 * or FNO_ERR_CUDA when a kernel found its shared-memory window misaligned
 * (the codes of fno_workspace_status). */
int fno_static_status(void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FNO_GB300_FNO_H_ */
