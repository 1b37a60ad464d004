// Internal declarations shared by the CUDA translation units of libctrecon.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ctrecon.h"

namespace ctr {

constexpr int MAX_BP_GROUPS = 8;   // angle groups of the backprojection (partial images)

// ---------------------------------------------------------------------------
// Error reporting (thread-local message, returned through ctr_last_error()).
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
ctr_status fail(ctr_status st, const std::string &msg);
ctr_status cuda_fail(cudaError_t e, const char *what);

#define CTR_CUDA(call)                                              \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return ::ctr::cuda_fail(e_, #call);  \
    } while (0)

// A named NVTX range over the enclosing scope (profilers group the kernels of each ABI
// call and solver phase by it; without a tool attached it costs a function call).
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};
#define CTR_NVTX_CAT2(a, b) a##b
#define CTR_NVTX_CAT(a, b) CTR_NVTX_CAT2(a, b)
#define CTR_NVTX(name) ::ctr::NvtxScope CTR_NVTX_CAT(nvtx_scope_, __LINE__)(name)

#define CTR_CHECK_LAUNCH(what)                                      \
    do {                                                            \
        cudaError_t e_ = cudaGetLastError();                        \
        if (e_ != cudaSuccess) return ::ctr::cuda_fail(e_, what);   \
    } while (0)

// Programmatic dependent launch.  A kernel launched by launch_pdl(true, ...) may be
// scheduled while the kernel before it in the stream is still running: it executes
// pdl_wait() before its first global-memory access, which returns once that kernel has
// completed and its writes are visible (and, since that kernel did the same, every
// earlier one).  pdl_trigger() lets the next such launch be scheduled as soon as every CTA
// of this grid is resident, so the launch latency overlaps the tail of this kernel.
// Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// The dynamic shared-memory limit is an attribute of the kernel function for the
// whole process, shared by every plan: only ever raise it.  (Its default is 48 KB minus
// the kernel's static shared memory, so the check is against the attribute itself.)
template <typename K>
inline ctr_status raise_smem_limit(K *kernel, size_t bytes)
{
    cudaFuncAttributes a;
    CTR_CUDA(cudaFuncGetAttributes(&a, (const void *)kernel));
    if ((size_t)a.maxDynamicSharedSizeBytes >= bytes) return CTR_OK;
    CTR_CUDA(cudaFuncSetAttribute((const void *)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return CTR_OK;
}

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

// ---------------------------------------------------------------------------
// Fixed-point detector geometry.
// The detector coordinate of pixel (i, j) at angle l, in bin units,
//     p = (x_i cos theta_l + y_j sin theta_l)/ds + (M-1)/2,
// is represented exactly as the integer P = i*C + j*S + O in units of 2^-F bins,
// with C = round(2^F h cos/ds), S = round(2^F h sin/ds) and O chosen so that the
// grid is centred.  floor(p) = P >> F and frac(p) = (P mod 2^F) 2^-F.  Both
// projectors derive every interpolation weight from the same integer P, so the
// ray-driven R_h is the exact transpose of the pixel-driven R_h^*.
// F = 32 for FP32/BF16 (weight = top 23 fraction bits), F = 48 or less for FP64.
// ---------------------------------------------------------------------------
struct AngleGeom {
    long long C, S, O;
};

// Ray-driven march of one angle: pixels are addressed by a "pick" index q along
// the axis where p changes fastest and a "march" index m along the other, with
// P(q, m) = q*A + m*B + Op, A > 0 and |B| <= A.  layout 0: q = i, m = j, values read
// from the transposed image uT[j][i]; layout 1: q = j, m = i, read from u[i][j].
// flip: the physical pick index is n-1-q.
struct AngleMarch {
    long long A, B, Op;
    int layout, flip;
    float kA;     // 2^F / A
    float oA;     // Op / A
    float binv;   // A / B (0 when |B/A| < 1e-9: rays parallel to the march axis)
};

// A job of the forward projector's symmetric path.  The fixed-point geometry is
// exactly invariant under the symmetries of the pixel grid: an angle whose (C, S) is
// (a, b), (-a, b), (b, a) or (-b, a) has P_l(i, j) = P_c(T(i, j)) for the canonical
// pair (a, b), a >= b >= 0, with T = id, (n-1-i, j), (j, i), (j, n-1-i).  One ray
// march of (a, b) over the "orbit image" (channel v at march pixel (q, m) holds
// u(T_v^{-1}(q, m))) therefore serves up to four angles.
struct OrbitJob {
    AngleMarch am;                // canonical march: layout 0, flip 0, A = a, B = b
    alignas(16) int l[4];         // angle of each channel (-1: none)
};

// Kernel-side parameter blocks ------------------------------------------------
template <typename T>
struct BackprojEpi {
    T *out;            // real output (n*n) or complex output (n*n pairs) when complex_out
    int complex_out;
    T scale;           // multiplies the backprojection sum
    const T *px;       // optional vector field (x plane, y plane = px + n*n) for -tau div
    T divtau;          // coefficient of div p (value = scale*R^*g - divtau*div p)
    T outscale;        // final multiplier
    T inv_h;
    const T *ub, *uu;  // optional: value += ub - uu (Alg. 5: bar u - u), or += ub when uu is null
    T *bar_out;        // optional (Alg. 1): bar_out = 2 value - ub (the extrapolated iterate)
};

// div_h p at pixel (i, j): (d1 + d2)/h, backward differences with Dirichlet ends
// (Sec. 3.1); px holds the x plane, px + n*n the y plane.
template <typename T>
__device__ __forceinline__ T div_at(const T *__restrict__ px, int n, int i, int j, T inv_h)
{
    if (n < 2) return T(0);
    const T *py = px + (size_t)n * n;
    T d1, d2;
    if (i == 0) d1 = px[j];
    else if (i == n - 1) d1 = -px[(size_t)(n - 2) * n + j];
    else d1 = px[(size_t)i * n + j] - px[(size_t)(i - 1) * n + j];
    const size_t row = (size_t)i * n;
    if (j == 0) d2 = py[row];
    else if (j == n - 1) d2 = -py[row + n - 2];
    else d2 = py[row + j] - py[row + j - 1];
    return (d1 + d2) * inv_h;
}

// The backprojection epilogue at pixel (i, j) for the sum acc:
// outscale (scale acc - divtau div p) [+ ub - uu].
template <typename T>
__device__ __forceinline__ T bp_epilogue_value(const BackprojEpi<T> &epi, int n, int i, int j, T acc)
{
    T v = acc * epi.scale;
    if (epi.px) v -= epi.divtau * div_at(epi.px, n, i, j, epi.inv_h);
    v *= epi.outscale;
    if (epi.ub) {
        const size_t e = (size_t)i * n + j;
        v += epi.ub[e] - (epi.uu ? epi.uu[e] : T(0));
    }
    return v;
}

// The fold of the symmetric backprojection (OrbitJob path): its partial planes
// [group][v][row][col] summed at image pixel (i, j) in a fixed order.
__device__ __forceinline__ float orbit_fold(const float *__restrict__ part, int groups, int n, int i, int j)
{
    const size_t nn = (size_t)n * n;
    const size_t e = (size_t)i * n + j, em = (size_t)(n - 1 - i) * n + j;
    float s = 0.f;
    for (int z = 0; z < groups; ++z) {
        const float *pz = part + (size_t)z * 4 * nn;
        s += pz[e] + pz[nn + em] + pz[2 * nn + e] + pz[3 * nn + em];
    }
    return s;
}

// Row and column of the flat pixel index e of an n-wide image in 32-bit arithmetic (every
// plan has n^2 < 2^32; a size_t division is a much longer instruction sequence).
__device__ __forceinline__ int pix_i(size_t e, int n) { return (int)((unsigned)e / (unsigned)n); }
__device__ __forceinline__ int pix_j(size_t e, int n) { return (int)((unsigned)e % (unsigned)n); }

// The same fold for the four adjacent pixels (i, col .. col + 3) (col and n multiples of 4)
// with 16-byte loads; each pixel's sum in the order of orbit_fold.
__device__ __forceinline__ float4 orbit_fold4(const float *__restrict__ part, int groups, int n, int i, int col)
{
    const size_t nn = (size_t)n * n;
    const size_t e = (size_t)i * n + col, em = (size_t)(n - 1 - i) * n + col;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int z = 0; z < groups; ++z) {
        const float *pz = part + (size_t)z * 4 * nn;
        const float4 a = __ldg(reinterpret_cast<const float4 *>(pz + e));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(pz + nn + em));
        const float4 c = __ldg(reinterpret_cast<const float4 *>(pz + 2 * nn + e));
        const float4 d = __ldg(reinterpret_cast<const float4 *>(pz + 3 * nn + em));
        s.x += a.x + b.x + c.x + d.x;
        s.y += a.y + b.y + c.y + d.y;
        s.z += a.z + b.z + c.z + d.z;
        s.w += a.w + b.w + c.w + d.w;
    }
    return s;
}

// grad_h u at pixel (i, j): forward differences with Neumann boundary (Sec. 3.1)
template <typename T>
__device__ __forceinline__ void grad_at(const T *__restrict__ u, int n, int i, int j, T inv_h, T &gx, T &gy)
{
    const size_t e = (size_t)i * n + j;
    const T c = u[e];
    gx = (i < n - 1) ? (u[e + n] - c) * inv_h : T(0);
    gy = (j < n - 1) ? (u[e + 1] - c) * inv_h : T(0);
}

// Step D of Alg. 4 at one pixel: TV dual update with the projection onto the ball of
// radius lam/tau, the next y2 = v2b + sigma tau grad u, optionally the certificate t2
// and (Alg. 5) bar u += max(2 u - bar u, 0) - u, the resolvent of I_{u >= 0}.
template <typename T>
struct TvDualJob {
    const T *u;
    int n;
    T sigma, tau, lam, inv_h;
    T *v2b, *y2, *t2, *ub;
};

template <typename T>
__device__ __forceinline__ void tv_dual_at(const TvDualJob<T> &t, int i, int j)
{
    const size_t nn = (size_t)t.n * t.n, e = (size_t)i * t.n + j;
    const T st = t.sigma * t.tau;
    T gx, gy;
    grad_at(t.u, t.n, i, j, t.inv_h, gx, gy);
    const T bx = t.v2b[e], by = t.v2b[e + nn];
    const T vx = bx + st * gx, vy = by + st * gy;
    const T zx = T(2) * vx - bx, zy = T(2) * vy - by;
    T tx = T(0), ty = T(0);
    if (t.lam > T(0)) {
        const T den = fmax(T(1), t.tau * sqrt(zx * zx + zy * zy) / t.lam);
        tx = zx / den;
        ty = zy / den;
    }
    const T nbx = bx + tx - vx, nby = by + ty - vy;
    t.v2b[e] = nbx;
    t.v2b[e + nn] = nby;
    t.y2[e] = nbx + st * gx;
    t.y2[e + nn] = nby + st * gy;
    if (t.t2) {
        t.t2[e] = tx;
        t.t2[e + nn] = ty;
    }
    if (t.ub) {
        const T uc = t.u[e], b0 = t.ub[e];
        t.ub[e] = b0 + fmax(T(2) * uc - b0, T(0)) - uc;
    }
}

template <typename T>
struct ForwardEpi {
    int mode;          // 0: plain g = scale*sum; 1: PDRQ dual step (Alg. 4); 2: CP dual step (Alg. 1);
                       // 3: Alg. 3 residual y1 = Rt u - a (and t1 = y1), Ru kept
    T *g;              // mode 0 output
    T scale;
    // mode 1
    T sigma;
    T *Ru;             // out: Rt u_new
    T *v1b;            // in/out: bar v1
    T *y1;             // out: bar v1_new + sigma Rt u_new
    __nv_bfloat16 *y1h;   // if set: y1 is stored here in bfloat16 instead (BF16 operand storage)
    T *t1;             // optional out: resolvent output (dual certificate)
    const T *dw, *da, *dlo, *dhi;   // per-bin data term, beta-scaled
};

// Radix sequence of the shared-memory Stockham FFT (product = n).
struct FftPasses {
    int count;
    int radix[16];
};

// One slice of a batch: everything a batched stage kernel needs (FP32).
struct SliceDesc {
    int n, N, M, wstride, bp_groups, per_group;
    int bp_tiles_x, bp_tiles_y;   // backprojection tiles
    int fwd_chunks;               // forward-projector CTAs per angle
    int rpc, cw;                  // FFT rows / columns per CTA
    int packed, prp, pcw;         // real-input FFT form (row pairs, n/2 + 1 columns): rows / columns per CTA
    const AngleGeom *geom;
    const AngleMarch *march;
    float2 *cbuf;
    const float2 *tw;
    const float *sym;
    FftPasses fp;
    float *u, *uT, *y1, *y2, *v2b, *bp_part;   // bp_part: angle-group images, or the symmetric planes
    int orbit;                    // symmetric projector path (per_group, bp_groups count jobs)
    int pair_jobs;                // the symmetric projectors' pair-job variants
    int twist;                    // the circulant preconditioner's 1-D transform in the column pass
    float *ub;                    // Alg. 5: bar u (updated by the TV stage); null for Alg. 4
    int n_jobs;
    const OrbitJob *jobs;
    float4 *ubar;
    BackprojEpi<float> bpe;       // step A epilogue
    ForwardEpi<float> fwe;        // step C epilogue
    float sigma, tau, lam, inv_h;
};

// Stages of one batched iteration (block counts per slice are prefix-summed).
// The angle-group sum / symmetric fold of the backprojection runs inside BS_FFT_ROWS;
// BS_BP_SYM, BS_ORBIT and BS_FWD_SYM serve the slices on the symmetric path, BS_BP and
// BS_FWD the others.
enum BatchStage { BS_BP = 0, BS_BP_SYM, BS_FFT_ROWS, BS_FFT_COLS, BS_FFT_ROWS_INV, BS_ORBIT, BS_FWD, BS_FWD_SYM,
                  BS_TV, BS_COUNT };

// Instantiated CUDA graphs kept across calls, keyed by everything the captured launches
// depend on (a tag for the loop, the block length, the scalar kernel arguments and the
// plan state that selects kernels); the buffers the kernels touch belong to the plan, so
// a replay with an equal key enqueues exactly the work a fresh capture would.  Least
// recently used entries are dropped beyond CAP.
struct GraphCache {
    struct Entry {
        std::vector<double> key;
        cudaGraphExec_t exec = nullptr;
        unsigned long long per_graph = 0;   // library kernels one replay launches
        unsigned long long last_use = 0;
    };
    static constexpr size_t CAP = 12;
    std::vector<Entry> entries;
    unsigned long long clock = 0;
    GraphCache() = default;
    GraphCache(const GraphCache &) = delete;
    GraphCache &operator=(const GraphCache &) = delete;
    ~GraphCache() { clear(); }
    void clear()
    {
        for (auto &e : entries)
            if (e.exec) cudaGraphExecDestroy(e.exec);
        entries.clear();
    }
};

// Grid barrier of the persistent batched iteration (device memory, zeroed before use).
struct GridBarrier {
    unsigned count;   // CTAs arrived at the current barrier
    unsigned gen;     // barriers completed
    int status;       // nonzero: a CTA's bounded wait ran out (the launch was abandoned)
    int pad;
};

// Diagnostics history of a solve with check_every > 0: one record of HIST_FIELDS doubles
// per check (beta, c, objective, data_fit, tv, violation, gap, dual_residual, rel_change,
// iters_done), at most MAX_CHECKS records per solve.
constexpr int HIST_FIELDS = 10;
constexpr int MAX_CHECKS = 4096;

}  // namespace ctr

// ---------------------------------------------------------------------------
// The plan.
// ---------------------------------------------------------------------------
constexpr int SYM_KEY_LEN = 8;   // sigma, tau, c, eps, nonneg, kind, kernel held, 1/h^2
struct ctr_plan {
    int n = 0, N = 0, M = 0;
    double h = 1.0, ds = 1.0;
    ctr_dtype dtype = CTR_F32;
    int F = 32;
    int device = 0;
    int wstride = 48;       // adjoint footprint stride (bins per staged angle)
    int ncand = 2;          // forward candidates per (ray, row)
    bool bf16 = false;      // CTR_BF16: projector operands stored in bfloat16, compute in FP32
    __nv_bfloat16 *uh = nullptr, *uTh = nullptr, *y1h = nullptr;   // bfloat16 operand copies
    int bp_groups = 1;      // angle groups of the backprojection (partial images summed)
    int bp_cap = 1;         // groups the partial-image workspace has room for
    void *bp_part = nullptr;   // bp_groups * n*n partial images (bp_groups > 1)
    std::vector<double> theta;
    std::vector<int> radices;    // FFT radices, product n
    bool fft_ok = false;         // n = 2^a 3^b (needed by the preconditioner only)
    size_t bytes = 0;
    std::vector<void *> allocations;
    mutable unsigned long long launches = 0;   // kernels launched (graph replays included)

    ctr::AngleGeom *d_geom = nullptr;
    ctr::AngleMarch *d_march = nullptr;
    bool orbit = false;                  // FP32 forward projector on the symmetric path
    int n_jobs = 0;
    ctr::OrbitJob *d_jobs = nullptr;
    void *ubar = nullptr;                // n*n float4 orbit image
    int obp_groups = 1;                  // job groups of the symmetric backprojection
    int pair_jobs = 0;                   // most jobs are pair jobs: both projectors take their pair variants
    int obp_cap = 1;                     // groups the partial-plane workspace has room for
    void *obp_part = nullptr;            // obp_groups * 4 * n*n partial planes
    void *d_twiddle = nullptr;  // n complex exp(-2 pi i t/n)

    // workspace, element type T (sizeof(T) = esize)
    size_t esize = 4;
    void *uT = nullptr;        // n*n
    void *cbuf = nullptr;      // n*n complex
    void *sym = nullptr;       // n*n preconditioner symbol (incl. 1/n^2)
    void *symh = nullptr;      // n*n sqrt(||xi||_eps)/n^2 for the power iteration
    void *u = nullptr;         // n*n primal iterate
    void *du = nullptr;        // n*n last increment / scratch
    void *x = nullptr;         // n*n power-iteration vector
    void *xt = nullptr;        // n*n scratch
    void *y2 = nullptr;        // 2*n*n
    void *v2b = nullptr;       // 2*n*n
    void *t2 = nullptr;        // 2*n*n
    void *y1 = nullptr;        // N*M
    void *Ru = nullptr;        // N*M
    void *v1b = nullptr;       // N*M
    void *t1 = nullptr;        // N*M
    void *ubar_u = nullptr;    // n*n bar u of Alg. 5 (non-negativity)
    int pdl = 1;               // programmatic dependent launch of the iteration's kernels
    int fft_form = 0;          // preconditioner passes: 0 warp-level where n allows (FP32, n = 256/512/1024), 1 CTA-level
    int precond_kind = 0;      // 0: inverse norm (Sec. 4.3.1); 1: impulse response; 2: circulant; 3: Richardson
    void *pk_s = nullptr;      // n*n DFT (2-D for kind 1, 1-D of the flattened image for kind 2) of the
                               // symmetrised impulse response of R_h^* R_h (built on first use)
    int pk_kind = 0;           // the kind pk_s currently holds (0: none)
    bool alg3 = false;         // the iteration is Alg. 3 (set for the duration of tv_pdrq2_solve)
    // the arguments sym / symh were last computed for (launch_symbols skips a repeat)
    mutable double sym_key[SYM_KEY_LEN] = {};
    mutable bool sym_valid = false;
    void *aux = nullptr;       // n*n image scratch (ADMM: the iterate before the last iteration)
    // detector-axis ramp filter: FFT length L >= 2M - 1 (2^a 3^b), its radices and
    // twiddles, and the real multiplier (the Ram-Lak kernel's DFT, times ds / L); the
    // tables are filled on first use
    int ramp_L = 0;
    std::vector<int> ramp_radices;
    void *d_ramp_tw = nullptr, *d_ramp_H = nullptr;
    bool ramp_ready = false;
    void *gs = nullptr;        // N*M scratch sinogram
    void *desc = nullptr;      // 4*N*M: w, a, lo, hi (beta-scaled)
    double *d_red = nullptr;   // reduction partials
    double *d_scal = nullptr;  // device scalars
    int red_blocks = 0;
    cudaStream_t stream = nullptr;       // internal stream (graph capture)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int fwd_slots = 1;                   // symmetric forward projector: adjacent jobs per CTA (1, 2, 4) ...
    int fwd_segs = 4;                    // ... and warps splitting a job's rows (2, 4, 8); see ctr_plan_set_fwd_shape
    int stg_wmax = 0;                    // staged forward shape (4, 1): widest window (pixels) ...
    int stg_nst = 0;                     // ... and most row blocks of one CTA
    double *d_hist = nullptr;            // MAX_CHECKS x HIST_FIELDS diagnostics records
    int hist_count = 0;                  // records the last solve wrote
    ctr::GraphCache graphs;              // instantiated iteration graphs, reused across calls
};

namespace ctr {

// Launch helpers implemented in the .cu files ------------------------------------
// defer_reduce with bp_groups > 1 (or on the symmetric path): only the partial
// images are written (bp_part, obp_part); the caller sums them (launch_circulant's
// bp_in).  bp_deferred(p) tells whether defer_reduce takes effect.
template <typename T>
ctr_status launch_backproject(const ctr_plan *p, const T *g, const BackprojEpi<T> &epi, cudaStream_t s,
                              bool defer_reduce = false);
// the same with the sinogram operand stored in bfloat16 (FP32 accumulation)
ctr_status launch_backproject_bf16(const ctr_plan *p, const __nv_bfloat16 *g, const BackprojEpi<float> &epi,
                                   cudaStream_t s, bool defer_reduce = false);
// the forward projector with the image operands stored in bfloat16 (FP32 accumulation)
ctr_status launch_forward_bf16(const ctr_plan *p, const __nv_bfloat16 *u, const __nv_bfloat16 *uT,
                               const ForwardEpi<float> &epi, cudaStream_t s);
// tv (optional, FP32 symmetric path only): the TV dual step of Alg. 4 fused into the
// kernel that builds the orbit image (both read u once)
template <typename T>
ctr_status launch_forward(const ctr_plan *p, const T *u, const T *uT, const ForwardEpi<T> &epi, cudaStream_t s,
                          const TvDualJob<T> *tv = nullptr);
template <typename T>
ctr_status launch_transpose(const ctr_plan *p, const T *in, T *out, cudaStream_t s);

// FFT-based circulant operators: out = F^{-1}(sym * F(in)) (sym includes 1/n^2).
// mode 0: out = result; mode 1: out += result (accumulate, solver update).
// outT (optional) receives the transpose of the final out; dout (optional) the
// result before accumulation.  bp_in (optional): the input is the backprojection
// left as angle-group partial images, or as the symmetric path's partial planes
// (launch_backproject with defer_reduce), summed and passed through *bp_in inside the
// first FFT pass.
template <typename T>
ctr_status launch_circulant(const ctr_plan *p, const T *in_real, bool in_is_cbuf, const T *sym, T *out,
                            int mode, T *outT, T *dout, cudaStream_t s, __nv_bfloat16 *outh = nullptr,
                            __nv_bfloat16 *outTh = nullptr, const BackprojEpi<T> *bp_in = nullptr);
template <typename T>
ctr_status launch_symbols(const ctr_plan *p, double sigma, double tau, double c, double eps, cudaStream_t s,
                          bool nonneg = false);
// cbuf = the 2-D forward DFT of the real n x n image in_real
template <typename T>
ctr_status launch_fft2_forward(const ctr_plan *p, const T *in_real, cudaStream_t s, bool twist = false);

template <typename T> ctr_status configure_radon(const ctr_plan *p);   // smem attributes, at plan creation
template <typename T> ctr_status configure_fft(const ctr_plan *p);
ctr_status fft_radices(int n, std::vector<int> &out);
int ramp_length(int M);   // smallest 2^a 3^b >= 2M - 1
// y = (ramp-filtered g) * outscale per view (N x M); yh (optional): the same in bfloat16 instead
template <typename T>
ctr_status launch_ramp(ctr_plan *p, const T *g, T *y, __nv_bfloat16 *yh, double outscale, cudaStream_t s);
size_t fft_smem_bytes(const ctr_plan *p, int which);

int backproject_tile_rows();   // pixel rows of a backprojection tile (its width is 32)
template <typename T> bool bp_deferred(const ctr_plan *p);
// false when the forward projector reads only u (the symmetric path builds its own
// orbit image): callers may then skip making the transposed copy uT
template <typename T> inline bool fwd_needs_transpose(const ctr_plan *p) { return !(sizeof(T) == 4 && p->orbit); }
int fwd_grid_x(int M);         // forward-projector grid: bin chunks
size_t stg_smem_bytes(int wmax, int nst_max, int rec_bytes);   // the staged forward projector's shared memory
constexpr size_t STG_SMEM_LIMIT = 227 * 1024;                   // dynamic shared memory one CTA may opt into
int stg_blocks_max(int n);
int stg_window(const std::vector<OrbitJob> &jobs, int n, int M);
int orbit_fwd_grid_y(int n_jobs);   // symmetric forward projector: job groups per bin chunk
int fwd_grid_y(int N);         // forward-projector grid: angle groups

// batched stages (one launch per stage over all slices of a batch)
size_t bp_smem_bytes(int wstride);
size_t obp_smem_bytes(int wstride, int jobs_per_group);   // the symmetric backprojection's dynamic shared memory
void bp_tiles(int n, int &tx, int &ty);
int fft_rows_per_cta(int n);
bool wfft_supported(const ctr_plan *p);        // the warp-level preconditioner passes apply
int fft_packed_rows_per_cta(const ctr_plan *p); // real-input form of the CTA-level passes: row pairs x 2 per CTA
int fft_packed_cols_per_cta(const ctr_plan *p); // ... stored columns per CTA
size_t fft_packed_smem(const ctr_plan *p, int which);   // ... dynamic shared memory (0 rows, 1 columns)
size_t fft_rows_smem(int n, size_t esize);   // dynamic shared memory of the row passes
size_t fft_cols_smem(int n, size_t esize);   // ... and of the column pass
int fft_cols_per_cta(int n, size_t esize);
ctr_status configure_batch_radon(size_t bp_smem, size_t obp_smem_max);
ctr_status configure_batch_fft(size_t rows_smem, size_t cols_smem);
ctr_status launch_batch_radon(int stage, const SliceDesc *sd, const int *prefix, int ns, int blocks, size_t smem,
                              cudaStream_t s);
ctr_status launch_batch_fft(int stage, const SliceDesc *sd, const int *prefix, int ns, int blocks, size_t smem,
                            cudaStream_t s);
ctr_status launch_batch_tv(const SliceDesc *sd, const int *prefix, int ns, int blocks, cudaStream_t s);
// the persistent form: one cooperative launch per iteration over every stage (kernels.cu)
int persist_blocks_per_sm(size_t smem);
ctr_status launch_batch_iteration(const SliceDesc *sd, const int *prefix, int ns, GridBarrier *gb,
                                  unsigned long long spin_limit, int grid, size_t smem, cudaStream_t s);

}  // namespace ctr

// A batch of independent slices (FP32), each with its own plan, solved together:
// every stage of an iteration is one launch over all slices.
struct ctr_batch {
    std::vector<ctr_plan *> plans;
    int device = 0;
    ctr::SliceDesc *d_desc = nullptr;   // one per slice
    int *d_prefix = nullptr;            // BS_COUNT x (slices + 1) block-offset tables
    int blocks[ctr::BS_COUNT] = {};
    size_t smem[ctr::BS_COUNT] = {};
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    unsigned long long launches = 0;
    ctr::GraphCache graphs;
    // iteration form: 0 = one launch per stage (graph-captured), 1 = one persistent
    // cooperative launch per iteration (k_batch_iteration)
    int mode = 0;
    int fft_packed = 1;                  // the stage tables use the real-input FFT form where slices allow it
    unsigned long long spin_limit = 1ull << 26;   // polls per grid barrier before giving up
    ctr::GridBarrier *d_gb = nullptr;
    int persist_grid = 0;                         // resident CTAs of the persistent kernel (0: unavailable)
    size_t persist_smem = 0;
};
