// fno_api.cu -- the C ABI of libfno: argument validation, workspace layout,
// the stage sequence of each operation, error reporting and launch timing.
//
// Stage sequence of the forward block (Alg. 2, Sec. IV-C of the paper):
//   tables -> fwd t,z (per column) -> fwd y -> fwd x -> mixing -> inv x -> inv y
//   -> inv z,t + epilogue
// The backward pass recomputes the forward spectrum from x (only the block
// input is kept between the passes) and runs the adjoint chain: the forward
// DFT kernels with the c(kt)/N-scaled t table produce G, the mixing adjoint
// gives dW and the input-spectrum gradient, and the inverse kernels with the
// unscaled t table bring it back to the grid.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "fno_internal.h"

namespace fno {

static thread_local std::string g_err;
static thread_local int g_status = FNO_OK;
static std::atomic<int64_t> g_launches{0};

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  g_status = code;
  return code;
}

static int cuda_fail(cudaError_t e, const char* where) {
  return fail(FNO_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// ---- launch timing ----------------------------------------------------------
struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
};
struct ProfAgg {
  std::string name;
  int64_t n;
  double ms;
};
static std::mutex g_prof_mu;
static bool g_prof = false;
static std::vector<ProfRec> g_recs;
static std::vector<cudaEvent_t> g_pool;
static size_t g_pool_used = 0;
static std::vector<ProfAgg> g_agg;

static cudaEvent_t pool_event() {
  if (g_pool_used == g_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g_pool.push_back(e);
  }
  return g_pool[g_pool_used++];
}

void prof_before(const char* name, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_prof) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEvent_t a = pool_event(), b = pool_event();
  if (!a || !b) return;
  cudaEventRecord(a, s);
  g_recs.push_back(ProfRec{name, a, b});
}

void prof_after(cudaStream_t s) {
  if (!g_prof) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_recs.empty()) cudaEventRecord(g_recs.back().b, s);
}

int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!cache[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 152;
    cache[dev] = n;
  }
  return cache[dev];
}

// ---- validation and workspace layout ---------------------------------------
static const int64_t kMaxChannels = 64;
static const int64_t kMaxModesT = 16;
static const size_t kMaxSmem = 227 * 1024;

static int to_dims(const fno_dims* dd, Dims* d) {
  if (!dd) return fail(FNO_ERR_INVALID_ARG, "dims is NULL");
  *d = Dims{dd->B, dd->C_in, dd->C_out, dd->Nx, dd->Ny, dd->Nz, dd->Nt,
            dd->mx, dd->my, dd->mz, dd->mt, 0, 0, 0, 0, 0, 0};
  if (d->B < 0) return fail(FNO_ERR_INVALID_ARG, "B = %lld < 0", (long long)d->B);
  const int64_t v[10] = {d->Ci, d->Co, d->Nx, d->Ny, d->Nz, d->Nt, d->mx, d->my, d->mz, d->mt};
  static const char* nm[10] = {"C_in", "C_out", "Nx", "Ny", "Nz", "Nt", "mx", "my", "mz", "mt"};
  for (int q = 0; q < 10; ++q)
    if (v[q] < 1) return fail(FNO_ERR_INVALID_ARG, "%s = %lld must be >= 1", nm[q], (long long)v[q]);
  for (int q = 2; q < 6; ++q)
    if (v[q] > (1 << 20)) return fail(FNO_ERR_INVALID_ARG, "%s = %lld too large", nm[q], (long long)v[q]);
  if (2 * d->mx > d->Nx) return fail(FNO_ERR_INVALID_ARG, "2*mx = %lld > Nx = %lld", (long long)(2 * d->mx), (long long)d->Nx);
  if (2 * d->my > d->Ny) return fail(FNO_ERR_INVALID_ARG, "2*my = %lld > Ny = %lld", (long long)(2 * d->my), (long long)d->Ny);
  if (2 * d->mz > d->Nz) return fail(FNO_ERR_INVALID_ARG, "2*mz = %lld > Nz = %lld", (long long)(2 * d->mz), (long long)d->Nz);
  if (d->mt > d->Nt / 2 + 1) return fail(FNO_ERR_INVALID_ARG, "mt = %lld > Nt/2 + 1 = %lld", (long long)d->mt, (long long)(d->Nt / 2 + 1));
  d->Jx = 2 * d->mx;
  d->Jy = 2 * d->my;
  d->Jz = 2 * d->mz;
  d->Jt = d->mt;
  d->Ng = d->Nx * d->Ny * d->Nz * d->Nt;
  d->Mk = d->Jx * d->Jy * d->Jz * d->Jt;
  return FNO_OK;
}

static bool is_tc(int precision) {
  return precision == FNO_BF16 || precision == FNO_BF16X3 || precision == FNO_TF32;
}
// split operands (hi + lo): split BF16, and TF32 (a TF32 value is exact in two BF16 parts)
static bool is_split(int precision) { return precision == FNO_BF16X3 || precision == FNO_TF32; }

static int check_support(const Dims& d, int precision, int op) {
  if (precision < FNO_FP32 || precision > FNO_BF16X3)
    return fail(FNO_ERR_INVALID_ARG, "precision %d is not an fno_precision", precision);
  if (op < FNO_OP_SPECTRAL_FWD || op > FNO_OP_BLOCK_TRAIN)
    return fail(FNO_ERR_INVALID_ARG, "op %d is not an fno_op", op);
  if (is_tc(precision)) {
    char why[256];
    if (!fwd_tz_mma_supported(d, why, sizeof(why))) return fail(FNO_ERR_UNSUPPORTED, "%s", why);
  }
  if (d.Ci > kMaxChannels || d.Co > kMaxChannels)
    return fail(FNO_ERR_UNSUPPORTED, "C_in, C_out must be <= %lld", (long long)kMaxChannels);
  // the inverse t stage of the epilogues keeps its factors in registers
  if (d.Jt > kMaxModesT)
    return fail(FNO_ERR_UNSUPPORTED, "mt = %lld must be <= %lld", (long long)d.Jt, (long long)kMaxModesT);
  const size_t need[5] = {
      fwd_tz_smem_bytes(d),
      line_smem_bytes((int)d.Ny, (int)d.Jy),
      line_smem_bytes((int)d.Nx, (int)d.Jx),
      line_smem_bytes((int)d.Jx, (int)d.Nx),
      line_smem_bytes((int)d.Jy, (int)d.Ny)};
  for (size_t q = 0; q < 5; ++q)
    if (need[q] > kMaxSmem)
      return fail(FNO_ERR_UNSUPPORTED, "grid/mode sizes need %zu bytes of shared memory in a DFT stage", need[q]);
  const int64_t Cm = d.Ci > d.Co ? d.Ci : d.Co;
  const bool bwd = (op == FNO_OP_BLOCK_BWD || op == FNO_OP_BLOCK_TRAIN);
  size_t e = epilogue_smem_bytes(d, bwd ? EPI_DA : EPI_FWD, (int)Cm, (int)Cm);
  if (e > kMaxSmem)
    return fail(FNO_ERR_UNSUPPORTED, "channel/grid sizes need %zu bytes of shared memory in the epilogue", e);
  if (op == FNO_OP_BLOCK_TRAIN) {
    const size_t p = pointwise_smem_bytes((int)d.Ci, (int)d.Co, true);
    if (p > kMaxSmem)
      return fail(FNO_ERR_UNSUPPORTED, "channel counts need %zu bytes of shared memory in the dA pass", p);
  }
  return FNO_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t err;  // device status word (nonzero: a bounded wait gave up)
  size_t tab[10];
  size_t t1, t2, xh, yh, gxh, da, part, mma_tab, tc_tab, gp, vz, total;  // vz 0: no region
  bool da_in_dx;
};

// Grids that the fused epilogues do not tile (Nt other than 16 and 32, or
// their other limits) take the synthesis path in the tensor-core precisions:
// the inverse z stage as a tensor-core line into V = [B Cs Nx Ny][Nz][Jt],
// the inverse t stage to real points (launch_synth_t) straight into the
// output, and the 1x1, bias and GELU in place (launch_pw_add).
static bool synth_shape_ok(const Dims& d, int64_t Cs, int64_t Cl) {
  return synth_t_supported((int)d.Nt, (int)d.Jt) && line_mma_supported((int)d.Jz, (int)d.Nz) &&
         Cs >= 1 && Cs <= 32 && (Cl == 0 || pw_add_supported((int)Cl, (int)Cs));
}
// whether a workspace for these sizes holds V: some epilogue mode of the block
// or the spectral convolution is then outside the mma.sync epilogue's tiling
static bool synth_region(const Dims& d) {
  const int Ci = (int)d.Ci, Co = (int)d.Co;
  if (!synth_shape_ok(d, Co, Ci) || !synth_shape_ok(d, Ci, Co)) return false;
  return !(epilogue_mma_supported(d, EPI_FWD, Co, Ci, nullptr, 0) &&
           epilogue_mma_supported(d, EPI_DX, Ci, Co, nullptr, 0) &&
           epilogue_mma_supported(d, EPI_SPECTRAL, Co, 0, nullptr, 0) &&
           epilogue_mma_supported(d, EPI_SPECTRAL, Ci, 0, nullptr, 0));
}

static Layout layout(const Dims& d, int op) {
  Layout L{};
  size_t off = 0;
  L.err = off;
  off += 256;
  const int64_t tsz[10] = {d.Jx * d.Nx, d.Jy * d.Ny, d.Jz * d.Nz, d.Jt * d.Nt, d.Jt * d.Nt,
                           d.Nx * d.Jx, d.Ny * d.Jy, d.Nz * d.Jz, d.Jt * d.Nt, d.Jt * d.Nt};
  for (int q = 0; q < 10; ++q) {
    L.tab[q] = off;
    off += align256(sizeof(float2) * (size_t)tsz[q]);
  }
  const int64_t Cm = d.Ci > d.Co ? d.Ci : d.Co;
  L.t1 = off;
  off += align256(sizeof(float2) * (size_t)(d.B * Cm * d.Nx * d.Ny * d.Jz * d.Jt));
  L.t2 = off;
  off += align256(sizeof(float2) * (size_t)(d.B * Cm * d.Nx * d.Jy * d.Jz * d.Jt));
  L.xh = off;
  off += align256(sizeof(float2) * (size_t)(d.B * d.Ci * d.Mk));
  L.yh = off;
  off += align256(sizeof(float2) * (size_t)(d.B * d.Co * d.Mk));
  // the training layout is the backward layout with GELU'(A) appended, so a
  // workspace sized for it serves both calls of a training step
  const bool block_bwd = (op == FNO_OP_BLOCK_BWD || op == FNO_OP_BLOCK_TRAIN);
  if (op == FNO_OP_SPECTRAL_BWD || block_bwd) {
    L.gxh = off;
    off += align256(sizeof(float2) * (size_t)(d.B * d.Ci * d.Mk));
  }
  if (block_bwd) {
    // dA lives in dx while dx is not yet written when the channel counts agree
    L.da_in_dx = (d.Ci == d.Co);
    if (!L.da_in_dx) {
      L.da = off;
      off += align256(sizeof(float) * (size_t)(d.B * d.Co * d.Ng));
    }
    L.part = off;
    const int rows = epilogue_max_grid();
    off += align256(sizeof(float) * (size_t)rows * (size_t)(d.Ci * d.Co + d.Co));
  }
  L.mma_tab = off;  // basis fragments of the mma.sync epilogue
  off += align256(epilogue_mma_table_bytes(d));
  L.tc_tab = off;  // z basis images of the tcgen05 epilogue
  off += align256(epilogue_tc_table_bytes(d));
  if (op == FNO_OP_BLOCK_TRAIN) {
    L.gp = off;  // GELU'(A) of the training forward, [B][C_out][grid]
    off += align256(sizeof(float) * (size_t)(d.B * d.Co * d.Ng));
  }
  if (synth_region(d)) {
    const int64_t Cm2 = d.Ci > d.Co ? d.Ci : d.Co;
    L.vz = off;  // inverse z stage of the synthesis path, [B Cm Nx Ny][Nz][Jt]
    off += align256(sizeof(float2) * (size_t)(d.B * Cm2 * d.Nx * d.Ny * d.Nz * d.Jt));
  }
  L.total = off;
  return L;
}

static Tables tables_at(char* ws, const Layout& L) {
  Tables T;
  float2** p[10] = {&T.Fx, &T.Fy, &T.Fz, &T.Ft, &T.Fta, &T.Ix, &T.Iy, &T.Iz, &T.Its, &T.Itu};
  for (int q = 0; q < 10; ++q) *p[q] = reinterpret_cast<float2*>(ws + L.tab[q]);
  return T;
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

static int check_ws(void* ws, size_t ws_bytes, const Layout& L) {
  if (ws_bytes < L.total)
    return fail(FNO_ERR_WORKSPACE, "workspace of %zu bytes < %zu required", ws_bytes, L.total);
  if (L.total > 0 && !ws) return fail(FNO_ERR_WORKSPACE, "workspace is NULL");
  if (ws && !aligned(ws, 256)) return fail(FNO_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  return FNO_OK;
}

#define REQ(ptr, al)                                                                  \
  do {                                                                                \
    if (!(ptr)) return fail(FNO_ERR_INVALID_ARG, "%s is NULL", #ptr);                \
    if (!aligned((ptr), (al))) return fail(FNO_ERR_INVALID_ARG, "%s must be %d-byte aligned", #ptr, (int)(al)); \
  } while (0)

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)


// One complex axis: mma.sync for the tensor-core precisions, FP32 otherwise.
static cudaError_t line(const float2* in, float2* out, int64_t outer, int nin, int nout, int64_t inner,
                        const float2* tab, int precision, cudaStream_t s) {
  if (is_tc(precision) && line_mma_supported(nin, nout))
    return launch_line_mma(in, out, outer, nin, nout, inner, tab, is_split(precision), precision == FNO_TF32, s);
  return launch_line_f32(in, out, outer, nin, nout, inner, tab, s);
}

// The y then x stages of a forward kept-mode spectrum, from the t, z spectra
// t1 = [B][C][Nx][Ny][Jz][Jt] into out.  Uses t2.
static int spectrum_yx(const Dims& d, int64_t C, const Tables& T, const float2* t1, float2* t2, float2* out,
                       cudaStream_t s, int precision) {
  CK(line(t1, t2, d.B * C * d.Nx, (int)d.Ny, (int)d.Jy, d.Jz * d.Jt, T.Fy, precision, s));
  CK(line(t2, out, d.B * C, (int)d.Nx, (int)d.Jx, d.Jy * d.Jz * d.Jt, T.Fx, precision, s));
  return FNO_OK;
}

// Forward kept-mode spectrum of C channels of src into out: t,z per column
// (tensor cores for the BF16 precisions) -> y -> x.  Uses t1, t2.
static int spectrum_f32(const Dims& d, int64_t C, const float* src, const float2* ft,
                        const Tables& T, float2* t1, float2* t2, float2* out, cudaStream_t s,
                        int precision = FNO_FP32, int* err = nullptr) {
  if (is_tc(precision))
    CK(launch_fwd_tz_mma(src, t1, d.B * C * d.Nx * d.Ny, d, ft, T.Fz, is_split(precision),
                         precision == FNO_TF32, err, s));
  else
    CK(launch_fwd_tz_f32(src, t1, d.B * C * d.Nx * d.Ny, d, ft, T.Fz, s));
  return spectrum_yx(d, C, T, t1, t2, out, s, precision);
}

// Inverse x then y of C channels of kept spectra into u1 = [B][C][Nx][Ny][Jz][Jt].
static int inverse_xy_f32(const Dims& d, int64_t C, const float2* sp, const Tables& T, float2* t2,
                          float2* u1, cudaStream_t s, int precision = FNO_FP32) {
  CK(line(sp, t2, d.B * C, (int)d.Jx, (int)d.Nx, d.Jy * d.Jz * d.Jt, T.Ix, precision, s));
  CK(line(t2, u1, d.B * C * d.Nx, (int)d.Jy, (int)d.Ny, d.Jz * d.Jt, T.Iy, precision, s));
  return FNO_OK;
}

// The synthesis path (see synth_shape_ok): the dX form writes its 1x1 term
// first, while dA (which may live in dx) is intact, and the inverse t stage
// adds to it; the forward writes S into z first and the pointwise pass reads
// it back as the summand of A.
static cudaError_t synth_epilogue(const Dims& d, const EpiArgs& a, int precision, float2* V,
                                  cudaStream_t s) {
  const int64_t cols = d.B * a.Cs * d.Nx * d.Ny;
  const bool dx = (a.mode == EPI_DX);
  if (dx) {
    cudaError_t e = launch_pw_add(a.lin_in, a.wlin, a.w_si, a.w_sc, nullptr, a.out, nullptr, d.B, d.Ng,
                                  a.Cl, a.Cs, false, s);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = line(a.U, V, cols, (int)d.Jz, (int)d.Nz, d.Jt, a.Iz, precision, s);
  if (e != cudaSuccess) return e;
  e = launch_synth_t(V, a.out, cols * d.Nz, (int)d.Nt, (int)d.Jt, a.It, dx, is_split(precision),
                     precision == FNO_TF32, s);
  if (e != cudaSuccess) return e;
  if (a.mode == EPI_FWD)
    return launch_pw_add(a.lin_in, a.wlin, a.w_si, a.w_sc, a.bias, a.out, a.gp, d.B, d.Ng, a.Cl, a.Cs, true,
                         s);
  return cudaSuccess;
}

// The fused inverse z, t + epilogue stage: split BF16 and TF32 on tcgen05 (TMEM
// accumulators) where its tiling applies, then warp-level mma.sync (plain BF16,
// the dA mode and the shapes tcgen05 does not tile), then, in the tensor-core
// precisions, the synthesis path for other Nt (not the dA mode), else FP32 on
// the CUDA cores (the plain form, and the exact fallback for other shapes).
static cudaError_t epilogue(const Dims& d, EpiArgs a, int precision, char* base, const Layout& L,
                            int* err, int* grid_used, cudaStream_t s) {
  // plain BF16 (one product, no split operands to build) measured faster on
  // mma.sync; the split precisions on tcgen05
  if (is_split(precision) && epilogue_tc_supported(d, a.mode, a.Cs, a.Cl, nullptr, 0))
    return launch_epilogue_tc(d, a, true, precision == FNO_TF32, base + L.tc_tab, err, s);
  if (is_tc(precision) && epilogue_mma_supported(d, a.mode, a.Cs, a.Cl, nullptr, 0))
    return launch_epilogue_mma(d, a, is_split(precision), precision == FNO_TF32, base + L.mma_tab, err,
                               grid_used, s);
  if (is_tc(precision) && a.mode != EPI_DA && L.vz != 0 && synth_shape_ok(d, a.Cs, a.Cl))
    return synth_epilogue(d, a, precision, reinterpret_cast<float2*>(base + L.vz), s);
  return launch_epilogue_f32(d, a, grid_used, s);
}

// Whether a training forward keeps GELU'(A) for the backward's dA pass.  The
// pass wins wherever it contracts dW_lin on the tensor cores, and over the FP32
// dA epilogue; with more channels than that in the tensor-core precisions, the
// tensor-core dA epilogue (A re-evaluated from the kept spectra) is the faster
// form, and the forward skips the store.
static bool keep_gelu_grad(const Dims& d, int precision) {
  if (pointwise_da_mma_fits((int)d.Ci, (int)d.Co)) return true;
  return !(is_tc(precision) &&
           epilogue_mma_supported(d, EPI_DA, (int)d.Co, (int)d.Ci, nullptr, 0));
}

static int forward_common(const Dims& d, int precision, int op, const float* x, const float* w,
                          const float* w_lin, const float* bias, float* out, void* ws,
                          size_t ws_bytes, cudaStream_t s) {
  int rc = check_support(d, precision, op);
  if (rc) return rc;
  const Layout L = layout(d, op);
  if ((rc = check_ws(ws, ws_bytes, L))) return rc;
  REQ(w, 8);
  const bool block = (op == FNO_OP_BLOCK_FWD || op == FNO_OP_BLOCK_TRAIN);
  if (block) {
    REQ(w_lin, 4);
    REQ(bias, 4);
  }
  if (d.B == 0) return FNO_OK;
  REQ(x, 16);
  REQ(out, 16);
  char* base = static_cast<char*>(ws);
  const Tables T = tables_at(base, L);
  float2* t1 = reinterpret_cast<float2*>(base + L.t1);
  float2* t2 = reinterpret_cast<float2*>(base + L.t2);
  float2* xh = reinterpret_cast<float2*>(base + L.xh);
  float2* yh = reinterpret_cast<float2*>(base + L.yh);
  int* err = reinterpret_cast<int*>(base + L.err);
  CK(launch_tables(d, T, err, s));
  if ((rc = spectrum_f32(d, d.Ci, x, T.Ft, T, t1, t2, xh, s, precision, err))) return rc;
  CK(launch_mix_f32(d, xh, reinterpret_cast<const float2*>(w), yh, s));
  if ((rc = inverse_xy_f32(d, d.Co, yh, T, t2, t1, s, precision))) return rc;
  EpiArgs a{};
  a.mode = block ? EPI_FWD : EPI_SPECTRAL;
  a.U = t1;
  a.lin_in = x;
  a.wlin = w_lin;
  a.bias = bias;
  a.out = out;
  a.gp = (op == FNO_OP_BLOCK_TRAIN && keep_gelu_grad(d, precision))
             ? reinterpret_cast<float*>(base + L.gp)
             : nullptr;
  a.Iz = T.Iz;
  a.It = T.Its;
  a.Cs = (int)d.Co;
  a.Cl = block ? (int)d.Ci : 0;
  a.w_si = (int)d.Co;
  a.w_sc = 1;
  CK(epilogue(d, a, precision, base, L, err, nullptr, s));
  return FNO_OK;
}

// ---- forward state kept in a workspace ---------------------------------------
// After fno_block_fwd the workspace holds the block input's kept spectrum X̂ and
// the inverse x, y partial U1 of the output spectrum (fno_block_fwd_train adds
// GELU'(A)); fno_block_bwd_saved reuses them instead of recomputing.  The
// library remembers, per workspace, which forward call left that state
// (host-side bookkeeping: no device sync); any other call on the workspace
// forgets it.
struct SavedFwd {
  const void* ws;
  const float* x;
  const float* w;
  fno_dims dims;
  int precision;
  bool train;  // GELU'(A) kept too
};
static std::mutex g_saved_mu;
static std::vector<SavedFwd> g_saved;
static const size_t kSavedMax = 4096;

static void saved_forget(const void* ws) {
  std::lock_guard<std::mutex> lk(g_saved_mu);
  for (size_t i = 0; i < g_saved.size(); ++i)
    if (g_saved[i].ws == ws) {
      g_saved.erase(g_saved.begin() + (long)i);
      return;
    }
}
static void saved_set(const void* ws, const float* x, const float* w, const fno_dims& dims,
                      int precision, bool train) {
  saved_forget(ws);
  std::lock_guard<std::mutex> lk(g_saved_mu);
  if (g_saved.size() >= kSavedMax) g_saved.erase(g_saved.begin());
  g_saved.push_back(SavedFwd{ws, x, w, dims, precision, train});
}
static bool saved_match(const void* ws, const float* x, const float* w, const fno_dims& dims,
                        int precision, bool* train) {
  std::lock_guard<std::mutex> lk(g_saved_mu);
  for (const SavedFwd& r : g_saved)
    if (r.ws == ws) {
      *train = r.train;
      return r.x == x && r.w == w && r.precision == precision &&
             std::memcmp(&r.dims, &dims, sizeof(fno_dims)) == 0;
    }
  return false;
}

// ---- layers around the blocks (Alg. 1) --------------------------------------
static int to_pw(const fno_pw_dims* pd, int64_t* B, int* Ci, int* Co, int64_t* P) {
  if (!pd) return fail(FNO_ERR_INVALID_ARG, "dims is NULL");
  if (pd->B < 0) return fail(FNO_ERR_INVALID_ARG, "B = %lld < 0", (long long)pd->B);
  if (pd->P < 0) return fail(FNO_ERR_INVALID_ARG, "P = %lld < 0", (long long)pd->P);
  if (pd->C_in < 1 || pd->C_in > kMaxChannels || pd->C_out < 1 || pd->C_out > kMaxChannels)
    return fail(FNO_ERR_INVALID_ARG, "C_in = %lld, C_out = %lld must lie in 1..%lld",
                (long long)pd->C_in, (long long)pd->C_out, (long long)kMaxChannels);
  if (pd->P > ((int64_t)1 << 40) || pd->B > ((int64_t)1 << 20))
    return fail(FNO_ERR_INVALID_ARG, "B = %lld, P = %lld too large", (long long)pd->B,
                (long long)pd->P);
  *B = pd->B;
  *Ci = (int)pd->C_in;
  *Co = (int)pd->C_out;
  *P = pd->P;
  return FNO_OK;
}

static size_t pw_ws_bytes(int Ci, int Co) {
  // per-CTA partial rows, then a db scratch for callers that pass db = NULL
  return align256(sizeof(float) * (size_t)pointwise_max_grid(Ci, Co) * (size_t)(Ci * Co + Co)) +
         align256(sizeof(float) * (size_t)Co);
}

}  // namespace fno

using namespace fno;

extern "C" {

size_t fno_workspace_bytes(const fno_dims* dims, int precision, int op) {
  Dims d;
  if (to_dims(dims, &d)) return 0;
  if (check_support(d, precision, op)) return 0;
  return layout(d, op).total;
}

int fno_spectral_fwd(const fno_dims* dims, int precision, const float* x, const float* w,
                     float* y, void* ws, size_t ws_bytes, void* stream) {
  Dims d;
  int rc = to_dims(dims, &d);
  if (rc) return rc;
  saved_forget(ws);
  return forward_common(d, precision, FNO_OP_SPECTRAL_FWD, x, w, nullptr, nullptr, y, ws,
                        ws_bytes, (cudaStream_t)stream);
}

int fno_block_fwd(const fno_dims* dims, int precision, const float* x, const float* w,
                  const float* w_lin, const float* bias, float* z, void* ws, size_t ws_bytes,
                  void* stream) {
  Dims d;
  int rc = to_dims(dims, &d);
  if (rc) return rc;
  saved_forget(ws);
  rc = forward_common(d, precision, FNO_OP_BLOCK_FWD, x, w, w_lin, bias, z, ws, ws_bytes,
                      (cudaStream_t)stream);
  if (rc == FNO_OK && d.B > 0) saved_set(ws, x, w, *dims, precision, false);
  return rc;
}

int fno_block_fwd_train(const fno_dims* dims, int precision, const float* x, const float* w,
                        const float* w_lin, const float* bias, float* z, void* ws,
                        size_t ws_bytes, void* stream) {
  Dims d;
  int rc = to_dims(dims, &d);
  if (rc) return rc;
  saved_forget(ws);
  rc = forward_common(d, precision, FNO_OP_BLOCK_TRAIN, x, w, w_lin, bias, z, ws, ws_bytes,
                      (cudaStream_t)stream);
  if (rc == FNO_OK && d.B > 0) saved_set(ws, x, w, *dims, precision, keep_gelu_grad(d, precision));
  return rc;
}

int fno_spectral_bwd(const fno_dims* dims, int precision, const float* x, const float* w,
                     const float* dy, float* dx, float* dw, void* ws, size_t ws_bytes,
                     void* stream) {
  Dims d;
  int rc = to_dims(dims, &d);
  if (rc) return rc;
  const int op = FNO_OP_SPECTRAL_BWD;
  saved_forget(ws);
  if ((rc = check_support(d, precision, op))) return rc;
  const Layout L = layout(d, op);
  if ((rc = check_ws(ws, ws_bytes, L))) return rc;
  if (!dx && !dw) return fail(FNO_ERR_INVALID_ARG, "dx and dw are both NULL");
  REQ(w, 8);
  if (dw && !aligned(dw, 8)) return fail(FNO_ERR_INVALID_ARG, "dw must be 8-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  if (d.B == 0) {
    if (dw) CK(launch_fill_zero(dw, 2 * d.Ci * d.Co * d.Mk, s));
    return FNO_OK;
  }
  REQ(dy, 16);
  if (dw) REQ(x, 16);
  if (dx) REQ(dx, 16);
  char* base = static_cast<char*>(ws);
  const Tables T = tables_at(base, L);
  float2* t1 = reinterpret_cast<float2*>(base + L.t1);
  float2* t2 = reinterpret_cast<float2*>(base + L.t2);
  float2* xh = reinterpret_cast<float2*>(base + L.xh);
  float2* g = reinterpret_cast<float2*>(base + L.yh);
  float2* gxh = reinterpret_cast<float2*>(base + L.gxh);
  int* err = reinterpret_cast<int*>(base + L.err);
  CK(launch_tables(d, T, err, s));
  if ((rc = spectrum_f32(d, d.Co, dy, T.Fta, T, t1, t2, g, s, precision, err))) return rc;
  if (dw)
    if ((rc = spectrum_f32(d, d.Ci, x, T.Ft, T, t1, t2, xh, s, precision, err))) return rc;
  CK(launch_mix_adjoint_f32(d, xh, reinterpret_cast<const float2*>(w), g,
                            reinterpret_cast<float2*>(dw), dx ? gxh : nullptr, s));
  if (dx) {
    if ((rc = inverse_xy_f32(d, d.Ci, gxh, T, t2, t1, s, precision))) return rc;
    EpiArgs a{};
    a.mode = EPI_SPECTRAL;
    a.U = t1;
    a.out = dx;
    a.Iz = T.Iz;
    a.It = T.Itu;
    a.Cs = (int)d.Ci;
    a.Cl = 0;
    CK(epilogue(d, a, precision, base, L, err, nullptr, s));
  }
  return FNO_OK;
}

static int block_bwd_impl(const fno_dims* dims, int precision, const float* x, const float* w,
                          const float* w_lin, const float* bias, const float* dz, float* dx,
                          float* dw, float* dw_lin, float* db, void* ws, size_t ws_bytes,
                          void* stream, bool saved) {
  Dims d;
  int rc = to_dims(dims, &d);
  if (rc) return rc;
  const int op = FNO_OP_BLOCK_BWD;
  if ((rc = check_support(d, precision, op))) return rc;
  const Layout L = layout(d, op);
  if ((rc = check_ws(ws, ws_bytes, L))) return rc;
  REQ(w, 8);
  REQ(w_lin, 4);
  REQ(bias, 4);
  REQ(dw, 8);
  REQ(dw_lin, 4);
  REQ(db, 4);
  cudaStream_t s = (cudaStream_t)stream;
  if (d.B == 0) {
    CK(launch_fill_zero(dw, 2 * d.Ci * d.Co * d.Mk, s));
    CK(launch_fill_zero(dw_lin, d.Ci * d.Co, s));
    CK(launch_fill_zero(db, d.Co, s));
    return FNO_OK;
  }
  REQ(x, 16);
  REQ(dz, 16);
  REQ(dx, 16);
  char* base = static_cast<char*>(ws);
  const Tables T = tables_at(base, L);
  float2* t1 = reinterpret_cast<float2*>(base + L.t1);
  float2* t2 = reinterpret_cast<float2*>(base + L.t2);
  float2* xh = reinterpret_cast<float2*>(base + L.xh);
  float2* yh = reinterpret_cast<float2*>(base + L.yh);
  float2* gxh = reinterpret_cast<float2*>(base + L.gxh);
  float* da = L.da_in_dx ? dx : reinterpret_cast<float*>(base + L.da);
  float* part = reinterpret_cast<float*>(base + L.part);
  const float2* wc = reinterpret_cast<const float2*>(w);

  int* err = reinterpret_cast<int*>(base + L.err);
  bool train = false;
  if (saved && !saved_match(ws, x, w, *dims, precision, &train))
    return fail(FNO_ERR_INVALID_ARG,
                "the workspace does not hold the state of an fno_block_fwd call with these "
                "dims, precision, x and w");
  const Layout LT = layout(d, FNO_OP_BLOCK_TRAIN);
  if (train && (rc = check_ws(ws, ws_bytes, LT))) return rc;
  saved_forget(ws);  // the steps below overwrite the forward state
  CK(launch_tables(d, T, err, s));
  if (!saved) {
    // recompute the forward spectrum and the spectral partial U1 of the output
    if ((rc = spectrum_f32(d, d.Ci, x, T.Ft, T, t1, t2, xh, s, precision, err))) return rc;
    CK(launch_mix_f32(d, xh, wc, yh, s));
    if ((rc = inverse_xy_f32(d, d.Co, yh, T, t2, t1, s, precision))) return rc;
  }
  int rows = 0;
  bool tz_done = false;  // t1 already holds the t, z spectrum of dA
  if (train) {
    const float* gp = reinterpret_cast<const float*>(base + LT.gp);
    if (is_tc(precision) && da_tz_supported(d, nullptr, 0)) {
      // dA = dz GELU'(A) with the partial sums of dW_lin and db and the t, z
      // DFT of dA, in one pass over x, dz and GELU'(A)
      CK(launch_da_tz(x, gp, dz, da, t1, part, epilogue_max_grid(), d, T.Fta, T.Fz, is_split(precision),
                      precision == FNO_TF32, err, &rows, s));
      tz_done = true;
    } else {
      // dA = dz GELU'(A) from the training forward's GELU'(A): one pointwise
      // pass with the partial sums of dW_lin and db
      CK(launch_pointwise_bwd_saved(x, gp, dz, da, part, epilogue_max_grid(), d.B, d.Ng, (int)d.Ci, (int)d.Co,
                                    &rows, s));
    }
  } else {
  // dA = dz GELU'(A) with the partial sums of dW_lin and db
  EpiArgs a{};
  a.mode = EPI_DA;
  a.U = t1;
  a.lin_in = x;
  a.wlin = w_lin;
  a.bias = bias;
  a.dz = dz;
  a.out = da;
  a.part = part;
  a.Iz = T.Iz;
  a.It = T.Its;
  a.Cs = (int)d.Co;
  a.Cl = (int)d.Ci;
  a.w_si = (int)d.Co;
  a.w_sc = 1;
  CK(epilogue(d, a, precision, base, L, err, &rows, s));
  }
  CK(launch_reduce_partials(part, rows, (int)d.Ci, (int)d.Co, dw_lin, db, s));
  // G = (c/N) DFT(dA); dW and the input-spectrum gradient
  if (tz_done)
    rc = spectrum_yx(d, d.Co, T, t1, t2, yh, s, precision);
  else
    rc = spectrum_f32(d, d.Co, da, T.Fta, T, t1, t2, yh, s, precision, err);
  if (rc) return rc;
  CK(launch_mix_adjoint_f32(d, xh, wc, yh, reinterpret_cast<float2*>(dw), gxh, s));
  // dX = inverse(GXh) + W_lin dA
  if ((rc = inverse_xy_f32(d, d.Ci, gxh, T, t2, t1, s, precision))) return rc;
  EpiArgs q{};
  q.mode = EPI_DX;
  q.U = t1;
  q.lin_in = da;
  q.wlin = w_lin;
  q.out = dx;
  q.Iz = T.Iz;
  q.It = T.Itu;
  q.Cs = (int)d.Ci;
  q.Cl = (int)d.Co;
  q.w_si = 1;
  q.w_sc = (int)d.Co;
  CK(epilogue(d, q, precision, base, L, err, nullptr, s));
  return FNO_OK;
}

int fno_block_bwd(const fno_dims* dims, int precision, const float* x, const float* w,
                  const float* w_lin, const float* bias, const float* dz, float* dx, float* dw,
                  float* dw_lin, float* db, void* ws, size_t ws_bytes, void* stream) {
  return block_bwd_impl(dims, precision, x, w, w_lin, bias, dz, dx, dw, dw_lin, db, ws, ws_bytes,
                        stream, false);
}

int fno_block_bwd_saved(const fno_dims* dims, int precision, const float* x, const float* w,
                        const float* w_lin, const float* bias, const float* dz, float* dx,
                        float* dw, float* dw_lin, float* db, void* ws, size_t ws_bytes,
                        void* stream) {
  return block_bwd_impl(dims, precision, x, w, w_lin, bias, dz, dx, dw, dw_lin, db, ws, ws_bytes,
                        stream, true);
}

size_t fno_pointwise_workspace_bytes(const fno_pw_dims* dims) {
  int64_t B, P;
  int Ci, Co;
  if (to_pw(dims, &B, &Ci, &Co, &P)) return 0;
  return pw_ws_bytes(Ci, Co);
}

int fno_pointwise_fwd(const fno_pw_dims* dims, int act, const float* x, const float* w,
                      const float* bias, float* y, void* stream) {
  int64_t B, P;
  int Ci, Co;
  int rc = to_pw(dims, &B, &Ci, &Co, &P);
  if (rc) return rc;
  if (act != FNO_ACT_NONE && act != FNO_ACT_GELU)
    return fail(FNO_ERR_INVALID_ARG, "act = %d is not FNO_ACT_NONE or FNO_ACT_GELU", act);
  REQ(w, 4);
  if (bias && !aligned(bias, 4)) return fail(FNO_ERR_INVALID_ARG, "bias must be 4-byte aligned");
  if (B * P == 0) return FNO_OK;
  REQ(x, 4);
  REQ(y, 4);
  CK(launch_pointwise_fwd(x, w, bias, y, B, P, Ci, Co, act, (cudaStream_t)stream));
  return FNO_OK;
}

int fno_pointwise_bwd(const fno_pw_dims* dims, int act, const float* x, const float* w,
                      const float* bias, const float* dy, float* dx, float* dw, float* db,
                      void* ws, size_t ws_bytes, void* stream) {
  int64_t B, P;
  int Ci, Co;
  int rc = to_pw(dims, &B, &Ci, &Co, &P);
  if (rc) return rc;
  if (act != FNO_ACT_NONE && act != FNO_ACT_GELU)
    return fail(FNO_ERR_INVALID_ARG, "act = %d is not FNO_ACT_NONE or FNO_ACT_GELU", act);
  REQ(w, 4);
  REQ(dw, 4);
  if (bias && !aligned(bias, 4)) return fail(FNO_ERR_INVALID_ARG, "bias must be 4-byte aligned");
  if (db && !aligned(db, 4)) return fail(FNO_ERR_INVALID_ARG, "db must be 4-byte aligned");
  if (dx && !aligned(dx, 4)) return fail(FNO_ERR_INVALID_ARG, "dx must be 4-byte aligned");
  const size_t need = pw_ws_bytes(Ci, Co);
  if (ws_bytes < need)
    return fail(FNO_ERR_WORKSPACE, "workspace of %zu bytes < %zu required", ws_bytes, need);
  if (!ws) return fail(FNO_ERR_WORKSPACE, "workspace is NULL");
  if (!aligned(ws, 256)) return fail(FNO_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  float* part = static_cast<float*>(ws);
  float* dbs = db ? db : reinterpret_cast<float*>(static_cast<char*>(ws) + need - align256(sizeof(float) * (size_t)Co));
  if (B * P == 0) {
    CK(launch_fill_zero(dw, (int64_t)Ci * Co, s));
    if (db) CK(launch_fill_zero(db, Co, s));
    return FNO_OK;
  }
  REQ(x, 4);
  REQ(dy, 4);
  int rows = 0;
  CK(launch_pointwise_bwd(x, w, bias, dy, dx, part, B, P, Ci, Co, act, &rows, s));
  CK(launch_reduce_partials(part, rows, Ci, Co, dw, dbs, s));
  return FNO_OK;
}

size_t fno_mse_workspace_bytes(int64_t n) {
  if (n < 1) {
    fail(FNO_ERR_INVALID_ARG, "n = %lld must be >= 1", (long long)n);
    return 0;
  }
  return align256(sizeof(float) * (size_t)mse_max_grid());
}

int fno_mse_loss(int64_t n, const float* y, const float* target, float* loss, float* dy,
                 void* ws, size_t ws_bytes, void* stream) {
  if (n < 1) return fail(FNO_ERR_INVALID_ARG, "n = %lld must be >= 1", (long long)n);
  REQ(y, 4);
  REQ(target, 4);
  REQ(loss, 4);
  if (dy && !aligned(dy, 4)) return fail(FNO_ERR_INVALID_ARG, "dy must be 4-byte aligned");
  const size_t need = align256(sizeof(float) * (size_t)mse_max_grid());
  if (ws_bytes < need)
    return fail(FNO_ERR_WORKSPACE, "workspace of %zu bytes < %zu required", ws_bytes, need);
  if (!ws) return fail(FNO_ERR_WORKSPACE, "workspace is NULL");
  if (!aligned(ws, 256)) return fail(FNO_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  CK(launch_mse(y, target, dy, n, loss, static_cast<float*>(ws), (cudaStream_t)stream));
  return FNO_OK;
}

int fno_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr,
                  float beta1, float beta2, float eps, int64_t step, void* stream) {
  if (n < 0) return fail(FNO_ERR_INVALID_ARG, "n = %lld < 0", (long long)n);
  if (step < 1) return fail(FNO_ERR_INVALID_ARG, "step = %lld must be >= 1", (long long)step);
  if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f))
    return fail(FNO_ERR_INVALID_ARG, "beta1 = %g, beta2 = %g must lie in [0, 1)", beta1, beta2);
  if (!(eps > 0.f) || !(lr >= 0.f))
    return fail(FNO_ERR_INVALID_ARG, "eps = %g must be > 0 and lr = %g >= 0", eps, lr);
  if (n == 0) return FNO_OK;
  REQ(param, 4);
  REQ(grad, 4);
  REQ(m, 4);
  REQ(v, 4);
  const double bc1 = 1.0 - std::pow((double)beta1, (double)step);
  const double bc2 = 1.0 - std::pow((double)beta2, (double)step);
  CK(launch_adam(param, grad, m, v, n, lr, beta1, beta2, eps, bc1, bc2, (cudaStream_t)stream));
  return FNO_OK;
}

// Reads the device status word at the start of a scratch area (a workspace or
// the static scratch) once `stream` has drained, and decodes it.
static int read_status_word(const void* word, cudaStream_t s) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, word, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(status)");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  if (h == 2) return fail(FNO_ERR_CUDA, "a kernel refused a misaligned shared-memory window");
  if (h != 0) return fail(FNO_ERR_TIMEOUT, "a bounded device-side wait gave up (status %d)", h);
  return FNO_OK;
}

int fno_workspace_status(const void* ws, void* stream) {
  if (!ws) return fail(FNO_ERR_INVALID_ARG, "ws is NULL");
  return read_status_word(ws, (cudaStream_t)stream);
}

const char* fno_last_error(void) { return g_err.c_str(); }

int fno_last_status(void) { return g_status; }

int fno_version(void) { return 101; }

int64_t fno_launch_count(void) { return g_launches.load(); }

int fno_profile_start(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_recs.clear();
  g_agg.clear();
  g_pool_used = 0;
  g_prof = true;
  return FNO_OK;
}

int fno_profile_stop(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof = false;
  g_agg.clear();
  for (const ProfRec& r : g_recs) {
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    bool found = false;
    for (ProfAgg& g : g_agg)
      if (g.name == r.name) {
        g.n += 1;
        g.ms += ms;
        found = true;
        break;
      }
    if (!found) g_agg.push_back(ProfAgg{r.name, 1, (double)ms});
  }
  g_recs.clear();
  g_pool_used = 0;
  return FNO_OK;
}

int fno_profile_count(void) { return (int)g_agg.size(); }

int fno_profile_entry(int i, const char** name, int64_t* launches, double* total_ms) {
  if (i < 0 || i >= (int)g_agg.size()) return fail(FNO_ERR_INVALID_ARG, "profile entry %d out of range", i);
  if (name) *name = g_agg[i].name.c_str();
  if (launches) *launches = g_agg[i].n;
  if (total_ms) *total_ms = g_agg[i].ms;
  return FNO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free spectral forward: the scratch is a fixed device array of this
// file instead of a caller workspace (for callers that may not allocate device
// memory; see include/fno.h).
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_fno_static_scratch[FNO_STATIC_SCRATCH_BYTES];

namespace fno {
static std::mutex g_static_mu;
static void* g_static_ptr[64] = {nullptr};

// Device address of the static scratch on the current device.  The array's host
// name is only a host-side stand-in, so the address is looked up once per
// device with that device current and cached.  The lookup also loads the
// library's device code on that device (modules load lazily), which is when
// the array's memory is committed.  A cached address does not survive a reset
// of the device (cudaDeviceReset): the entry points below must not be used
// across one.
static int static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(FNO_ERR_UNSUPPORTED, "device ordinal %d >= 64", dev);
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fno_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    if (!p) return fail(FNO_ERR_CUDA, "cudaGetSymbolAddress returned NULL for the static scratch");
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return FNO_OK;
}
}  // namespace fno

extern "C" int fno_static_prepare(void) {
  void* ws = nullptr;
  return fno::static_scratch(&ws);
}

extern "C" int fno_static_status(void* stream) {
  void* ws = nullptr;
  int rc = fno::static_scratch(&ws);
  if (rc) return rc;
  return read_status_word(ws, (cudaStream_t)stream);
}

extern "C" int fno_spectral_fwd_static(const fno_dims* dims, int precision, const float* x,
                                       const float* w, float* y, void* stream) {
  Dims d;
  int rc = to_dims(dims, &d);
  if (rc) return rc;
  if ((rc = check_support(d, precision, FNO_OP_SPECTRAL_FWD))) return rc;
  const size_t need = layout(d, FNO_OP_SPECTRAL_FWD).total;
  if (need > FNO_STATIC_SCRATCH_BYTES)
    return fail(FNO_ERR_UNSUPPORTED,
                "these sizes need %zu bytes of scratch; the static scratch holds %zu bytes "
                "(use fno_spectral_fwd with a workspace)",
                need, (size_t)FNO_STATIC_SCRATCH_BYTES);
  void* ws = nullptr;
  if ((rc = static_scratch(&ws))) return rc;
  return forward_common(d, precision, FNO_OP_SPECTRAL_FWD, x, w, nullptr, nullptr, y, ws,
                        FNO_STATIC_SCRATCH_BYTES, (cudaStream_t)stream);
}

