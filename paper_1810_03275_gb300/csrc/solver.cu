// Alg. 4 (PDRQS1) on the GPU: the fused pointwise kernels around the projectors,
// deterministic FP64 reductions, the power iterations, the diagnostics and the
// iteration driver (optionally captured as CUDA graphs).
//
// One iteration is four stream-ordered steps, all in this library's kernels:
//   A  u_tmp = -sigma ( Rt^* y1 - tau div y2 )        backprojection + div epilogue
//   B  u    += F^{-1}( F(u_tmp) m ),  uT = u^T          three FFT passes
//   C  Rt u, v1 = v1b + sigma Rt u, t1 = prox(2 v1 - v1b), v1b += t1 - v1,
//      y1 = v1b + sigma Rt u                            ray-driven projection + epilogue
//   D  g = grad u, v2 = v2b + sigma tau g, t2 = P(2 v2 - v2b), v2b += t2 - v2,
//      y2 = v2b + sigma tau g                           stencil kernel
// y1, y2 carry Alg. 4's "v1b + sigma R u" and "v2b + sigma tau grad u" into the
// next iteration, so R_h u is computed once per iteration (Sec. 4.4).
#include <cmath>

#include <algorithm>

#include "ctr_internal.cuh"

namespace ctr {

namespace {

constexpr int RED_THREADS = 256;

// ------------------------------------------------------------------------------
// elementwise kernels
// ------------------------------------------------------------------------------
template <typename T>
__global__ void k_make_desc(const T *__restrict__ f, const uint8_t *__restrict__ mask, size_t len, double delta,
                            double trace_ratio, double inv_beta, T *w, T *a, T *lo, T *hi)
{
    // problem (C_h) with the data tolerance: off the metal trace w = 1, a = f,
    // [f - delta, f + delta] (delta < 0: unbounded); on the trace w = 0,
    // [trace_ratio f, +inf).  All values divided by beta (Sec. 5.1 scaling).
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < len; r += (size_t)gridDim.x * blockDim.x) {
        const double fv = (double)f[r];
        const bool tr = mask && mask[r];
        if (tr) {
            w[r] = T(0);
            a[r] = T(0);
            lo[r] = (T)(trace_ratio * fv * inv_beta);
            hi[r] = (T)inf;
        } else {
            w[r] = T(1);
            a[r] = (T)(fv * inv_beta);
            lo[r] = (T)(delta >= 0 ? (fv - delta) * inv_beta : -inf);
            hi[r] = (T)(delta >= 0 ? (fv + delta) * inv_beta : inf);
        }
    }
}

template <typename T>
__global__ void k_scale_desc(const T *__restrict__ wi, const T *__restrict__ ai, const T *__restrict__ loi,
                             const T *__restrict__ hii, size_t len, double inv_beta, T *w, T *a, T *lo, T *hi)
{
    for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < len; r += (size_t)gridDim.x * blockDim.x) {
        w[r] = wi[r];
        a[r] = (T)((double)ai[r] * inv_beta);
        lo[r] = (T)((double)loi[r] * inv_beta);
        hi[r] = (T)((double)hii[r] * inv_beta);
    }
}

// y = a + s * b
template <typename T>
__global__ void k_axpy(const T *__restrict__ a, const T *__restrict__ b, T s, size_t len, T *y)
{
    for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < len; r += (size_t)gridDim.x * blockDim.x)
        y[r] = a[r] + s * b[r];
}

template <typename T>
__global__ void k_grad(const T *__restrict__ u, int n, T inv_h, T *px)
{
    const size_t nn = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        T gx, gy;
        grad_at(u, n, pix_i(e, n), pix_j(e, n), inv_h, gx, gy);
        px[e] = gx;
        px[e + nn] = gy;
    }
}

template <typename T>
__global__ void k_div(const T *__restrict__ px, int n, T inv_h, T *d)
{
    const size_t nn = (size_t)n * n;
    const T *py = px + nn;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const int i = pix_i(e, n), j = pix_j(e, n);
        T d1 = T(0), d2 = T(0);
        if (n >= 2) {
            d1 = (i == 0) ? px[e] : (i == n - 1 ? -px[e - n] : px[e] - px[e - n]);
            d2 = (j == 0) ? py[e] : (j == n - 1 ? -py[e - 1] : py[e] - py[e - 1]);
        }
        d[e] = (d1 + d2) * inv_h;
    }
}

// y2 = v2b + sigma tau grad u   (start of the iteration from a given state)
template <typename T>
__global__ void k_init_y2(const T *__restrict__ u, const T *__restrict__ v2b, int n, T st, T inv_h, T *y2)
{
    const size_t nn = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        T gx, gy;
        grad_at(u, n, pix_i(e, n), pix_j(e, n), inv_h, gx, gy);
        y2[e] = v2b[e] + st * gx;
        y2[e + nn] = v2b[e + nn] + st * gy;
    }
}

// Step D of Alg. 4: TV dual update with the projection onto the ball of radius lam/tau.
// ub (Alg. 5 only): bar u += max(2 u - bar u, 0) - u, the resolvent of I_{u >= 0}.
template <typename T>
__device__ __forceinline__ void tv_dual_body(const T *__restrict__ u, int n, T sigma, T tau, T lam, T inv_h, T *v2b,
                                             T *y2, T *t2, T *ub, int b, int nb)
{
    const size_t nn = (size_t)n * n;
    const TvDualJob<T> job{u, n, sigma, tau, lam, inv_h, v2b, y2, t2, ub};
    for (size_t e = b * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)nb * blockDim.x)
        tv_dual_at(job, pix_i(e, n), pix_j(e, n));
}

template <typename T>
__global__ void __launch_bounds__(256)
k_tv_dual(const T *__restrict__ u, int n, T sigma, T tau, T lam, T inv_h, T *v2b, T *y2, T *t2, T *ub)
{
    tv_dual_body<T>(u, n, sigma, tau, lam, inv_h, v2b, y2, t2, ub, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256)
k_tv_dual_batch(const SliceDesc *__restrict__ sd, const int *__restrict__ prefix, int ns)
{
    int lo = 0, hi = ns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const SliceDesc &d = sd[lo];
    tv_dual_body<float>(d.u, d.n, d.sigma, d.tau, d.lam, d.inv_h, d.v2b, d.y2, nullptr, d.ub, blockIdx.x - prefix[lo],
                        prefix[lo + 1] - prefix[lo]);
}

// Alg. 1, TV dual: w = P_lambda(w + tau grad u_bar) (ball of radius lambda).
template <typename T>
__global__ void __launch_bounds__(256)
k_cp_tv(const T *__restrict__ ub, int n, T tau, T lam, T inv_h, T *w)
{
    const size_t nn = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        T gx, gy;
        grad_at(ub, n, pix_i(e, n), pix_j(e, n), inv_h, gx, gy);
        const T zx = w[e] + tau * gx, zy = w[e + nn] + tau * gy;
        T tx = T(0), ty = T(0);
        if (lam > T(0)) {
            const T den = fmax(T(1), sqrt(zx * zx + zy * zy) / lam);
            tx = zx / den;
            ty = zy / den;
        }
        w[e] = tx;
        w[e + nn] = ty;
    }
}

// Impulse-response preconditioner set-up -------------------------------------------
template <typename T>
__global__ void k_set_one(T *x) { *x = T(1); }

// k(i, j) = (kt(i, j) + kt(-i, -j)) / 2 with kt the impulse response y moved from
// (c, c) to the origin (indices mod n): the point-symmetric kernel.
// flat != 0 (circulant preconditioner): the same on the image flattened as t = i + n j,
// k_t = (y_{(t + p) mod n^2} + y_{(p - t) mod n^2}) / 2 with p = c + n c, written back at
// the pixel (i, j) of t.
template <typename T>
__global__ void k_kernel_sym(const T *__restrict__ y, int n, int c, int flat, T *k)
{
    const size_t nn = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const int i = pix_i(e, n), j = pix_j(e, n);
        if (flat) {
            const long long N = (long long)nn, t = i + (long long)n * j, pc = c + (long long)n * c;
            const long long ta = (t + pc) % N, tb = ((pc - t) % N + N) % N;
            const int ia = (int)(ta % n), ja = (int)(ta / n), ib = (int)(tb % n), jb = (int)(tb / n);
            k[e] = T(0.5) * (y[(size_t)ia * n + ja] + y[(size_t)ib * n + jb]);
            continue;
        }
        const int ia = (i + c) % n, ja = (j + c) % n;
        const int ib = ((c - i) % n + n) % n, jb = ((c - j) % n + n) % n;
        k[e] = T(0.5) * (y[(size_t)ia * n + ja] + y[(size_t)ib * n + jb]);
    }
}

// max over the real parts (the maximum is positive: it is at least the DC value, the
// sum of the kernel); positive doubles order like their bit patterns
template <typename T2>
__global__ void k_real_max(const T2 *__restrict__ F, size_t len, unsigned long long *mx)
{
    double m = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
        m = fmax(m, (double)F[e].x);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(mx, (unsigned long long)__double_as_longlong(m));
}

template <typename T, typename T2>
__global__ void k_real_floor(const T2 *__restrict__ F, size_t len, const unsigned long long *__restrict__ mx,
                             double floor_frac, T *s)
{
    const double lo = floor_frac * __longlong_as_double((long long)*mx);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
        s[e] = (T)fmax((double)F[e].x, lo);
}

__global__ void k_to_bf16(const float *__restrict__ x, size_t len, __nv_bfloat16 *y)
{
    for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < len; r += (size_t)gridDim.x * blockDim.x)
        y[r] = __float2bfloat16_rn(x[r]);
}

// Power-iteration start pattern x_ij = frac(1/2 + i/g + j/g^2) - 1/2, g the plastic number.
template <typename T>
__global__ void k_start_pattern(T *x, int n)
{
    const double g = 1.32471795724474602596;
    const size_t nn = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const double i = (double)(e / n), j = (double)(e % n);
        const double v = 0.5 + i / g + j / (g * g);
        x[e] = (T)(v - floor(v) - 0.5);
    }
}

// A block-uniform value evaluated once by thread 0 and broadcast through shared memory:
// FP64 arithmetic (a square root, a division) runs at a small fraction of the FP32 rate
// on this GPU, so a per-thread evaluation of a uniform FP64 expression costs more than the
// kernel's own work.
template <typename T, typename F>
__device__ __forceinline__ T block_uniform(F f)
{
    __shared__ T s_val;
    if (threadIdx.x == 0) s_val = f();
    __syncthreads();
    return s_val;
}

// x = y / sqrt(scal[idx])   (scal holds a squared norm)
template <typename T>
__global__ void k_normalize(const T *__restrict__ y, size_t len, const double *__restrict__ scal, int idx, T *x)
{
    pdl_wait();
    pdl_trigger();
    const T inv = block_uniform<T>([&] {
        const double s = scal[idx];
        return s > 0 ? (T)(1.0 / sqrt(s)) : T(0);
    });
    for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < len; r += (size_t)gridDim.x * blockDim.x)
        x[r] = y[r] * inv;
}

// ------------------------------------------------------------------------------
// deterministic reductions: each block writes NV partials; one block combines them
// ------------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], unsigned maxmask, double *out)
{
    __shared__ double sh[NV][RED_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_down_sync(0xffffffffu, x, o);
            x = ((maxmask >> q) & 1u) ? fmax(x, y) : x + y;
        }
        if (lane == 0) sh[q][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double x = sh[q][0];
            for (int w = 1; w < RED_THREADS / 32; ++w) x = ((maxmask >> q) & 1u) ? fmax(x, sh[q][w]) : x + sh[q][w];
            out[q] = x;
        }
    }
}

template <int NV>
__global__ void __launch_bounds__(RED_THREADS) k_finalize(const double *__restrict__ part, int nblk, unsigned maxmask, double *out)
{
    pdl_wait();
    pdl_trigger();
    double v[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = ((maxmask >> q) & 1u) ? -INFINITY : 0.0;
    for (int b = threadIdx.x; b < nblk; b += RED_THREADS)
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const double x = part[(size_t)b * NV + q];
            v[q] = ((maxmask >> q) & 1u) ? fmax(v[q], x) : v[q] + x;
        }
    block_reduce<NV>(v, maxmask, out);
}

// (sum a*b, sum b*b)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_dot2(const T *__restrict__ a, const T *__restrict__ b, size_t len, double *part)
{
    pdl_wait();
    pdl_trigger();
    double v[2] = {0.0, 0.0};
    for (size_t r = blockIdx.x * (size_t)RED_THREADS + threadIdx.x; r < len; r += (size_t)gridDim.x * RED_THREADS) {
        const double x = (double)a[r], y = (double)b[r];
        v[0] += x * y;
        v[1] += y * y;
    }
    block_reduce<2>(v, 0u, part + (size_t)blockIdx.x * 2);
}

// conjugate of the per-bin data term (beta-scaled values)
__device__ __forceinline__ double conj_term(double t, double w, double a, double lo, double hi)
{
    if (w > 0) {
        const double z = fmin(fmax(a + t / w, lo), hi);
        return t * z - 0.5 * w * (z - a) * (z - a);
    }
    if (t > 0) return t * hi;
    if (t < 0) return t * lo;
    return 0.0;
}

// sinogram diagnostics: sum 1/2 w (Ru - a)^2, max violation, sum of the data part of the gap
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
k_diag_sino(const T *__restrict__ Ru, const T *__restrict__ dw, const T *__restrict__ da, const T *__restrict__ dlo,
            const T *__restrict__ dhi, const T *__restrict__ t1, size_t len, double *part)
{
    double v[3] = {0.0, 0.0, 0.0};
    for (size_t r = blockIdx.x * (size_t)RED_THREADS + threadIdx.x; r < len; r += (size_t)gridDim.x * RED_THREADS) {
        const double z = Ru[r], w = dw[r], a = da[r], lo = dlo[r], hi = dhi[r];
        const double q = 0.5 * w * (z - a) * (z - a);
        v[0] += q;
        v[1] = fmax(v[1], fmax(lo - z, z - hi));
        if (t1) {
            const double t = t1[r];
            v[2] += q + conj_term(t, w, a, lo, hi) - z * t;
        }
    }
    block_reduce<3>(v, 2u, part + (size_t)blockIdx.x * 3);
}

// image diagnostics: TV(u), TV part of the gap, ||du||^2, ||u||^2
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
k_diag_img(const T *__restrict__ u, const T *__restrict__ du, const T *__restrict__ t2, int n, double inv_h,
           double lam, double tau, double *part)
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const size_t nn = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)RED_THREADS + threadIdx.x; e < nn; e += (size_t)gridDim.x * RED_THREADS) {
        const int i = pix_i(e, n), j = pix_j(e, n);
        const double c = u[e];
        const double gx = (i < n - 1) ? ((double)u[e + n] - c) * inv_h : 0.0;
        const double gy = (j < n - 1) ? ((double)u[e + 1] - c) * inv_h : 0.0;
        const double mag = sqrt(gx * gx + gy * gy);
        v[0] += mag;
        if (t2) v[1] += lam * mag - tau * (gx * (double)t2[e] + gy * (double)t2[e + nn]);
        if (du) v[2] += (double)du[e] * (double)du[e];
        v[3] += c * c;
    }
    block_reduce<4>(v, 0u, part + (size_t)blockIdx.x * 4);
}

inline int grid_for(size_t len, int threads = 256, int cap = 2048)
{
    size_t b = (len + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (size_t)cap) b = cap;
    return (int)b;
}

}  // namespace

// ------------------------------------------------------------------------------
// host-side building blocks
// ------------------------------------------------------------------------------
template <typename T>
ctr_status dot2(ctr_plan *p, const T *a, const T *b, size_t len, double *out_dev, cudaStream_t s)
{
    const int nb = grid_for(len, RED_THREADS * 8, p->red_blocks);   // 8 elements per thread: fewer FP64 tree adds
    p->launches++;
    launch_pdl(p->pdl != 0, k_dot2<T>, dim3(nb), dim3(RED_THREADS), 0, s, a, b, len, p->d_red);
    p->launches++;
    launch_pdl(p->pdl != 0, k_finalize<2>, dim3(1), dim3(RED_THREADS), 0, s, (const double *)p->d_red, nb, 0u, out_dev);
    CTR_CHECK_LAUNCH("k_dot2");
    return CTR_OK;
}

template <typename T>
ctr_status op_grad(ctr_plan *p, const T *u, T *px, cudaStream_t s)
{
    const size_t nn = (size_t)p->n * p->n;
    p->launches++;
    k_grad<T><<<grid_for(nn), 256, 0, s>>>(u, p->n, (T)(1.0 / p->h), px);
    CTR_CHECK_LAUNCH("k_grad");
    return CTR_OK;
}

template <typename T>
ctr_status op_div(ctr_plan *p, const T *px, T *d, cudaStream_t s)
{
    const size_t nn = (size_t)p->n * p->n;
    p->launches++;
    k_div<T><<<grid_for(nn), 256, 0, s>>>(px, p->n, (T)(1.0 / p->h), d);
    CTR_CHECK_LAUNCH("k_div");
    return CTR_OK;
}

// g = scale * R_h x  (x, xT both given)
template <typename T>
ctr_status op_forward(ctr_plan *p, const T *x, const T *xT, T *g, double scale, cudaStream_t s)
{
    ForwardEpi<T> e{};
    e.mode = 0;
    e.g = g;
    e.scale = (T)scale;
    return launch_forward<T>(p, x, xT, e, s);
}

// u = scale * R_h^* g
template <typename T>
ctr_status op_adjoint(ctr_plan *p, const T *g, T *u, double scale, cudaStream_t s)
{
    BackprojEpi<T> e{};
    e.out = u;
    e.complex_out = 0;
    e.scale = (T)scale;
    e.px = nullptr;
    e.divtau = T(0);
    e.outscale = T(1);
    e.inv_h = (T)(1.0 / p->h);
    return launch_backproject<T>(p, g, e, s);
}

// BF16 operand storage: g = R_h u with u, uT in bfloat16; u = R_h^* g with g in bfloat16
// (FP32 accumulation, FP32 results)
ctr_status op_forward_bf16(ctr_plan *p, const __nv_bfloat16 *u, const __nv_bfloat16 *uT, float *g, cudaStream_t s)
{
    ForwardEpi<float> e{};
    e.mode = 0;
    e.g = g;
    e.scale = 1.f;
    return launch_forward_bf16(p, u, uT, e, s);
}

ctr_status op_adjoint_bf16(ctr_plan *p, const __nv_bfloat16 *g, float *u, cudaStream_t s)
{
    BackprojEpi<float> e{};
    e.out = u;
    e.scale = 1.f;
    e.outscale = 1.f;
    e.inv_h = (float)(1.0 / p->h);
    return launch_backproject_bf16(p, g, e, s);
}

// `count` calls of step() on stream s, blk at a time replayed from one captured CUDA
// graph (blk <= 0 or count < blk: plain launches).  step() must enqueue the same work on
// every call.  With a key the instantiated graph stays in `cache` and later calls with an
// equal key replay it without capturing again (the key must hold every argument of the
// captured launches that can change between calls; buffers are fixed per plan).
// `launches` counts this library's kernels (graph replays included).
template <typename F>
ctr_status run_graphed_in(GraphCache &cache, unsigned long long &launches, int count, int blk, F &&step,
                          cudaStream_t s, const std::vector<double> *key)
{
    ctr_status st = CTR_OK;
    int done = 0;
    if (blk > 0 && count >= blk) {
        GraphCache::Entry *hit = nullptr;
        if (key)
            for (auto &e : cache.entries)
                if (e.key == *key) {
                    hit = &e;
                    break;
                }
        cudaGraphExec_t exec = nullptr;
        unsigned long long per_graph = 0;
        if (hit) {
            exec = hit->exec;
            per_graph = hit->per_graph;
            hit->last_use = ++cache.clock;
        } else {
            cudaGraph_t graph = nullptr;
            const unsigned long long before = launches;
            CTR_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            for (int k = 0; k < blk && st == CTR_OK; ++k) st = step();
            cudaError_t ce = cudaStreamEndCapture(s, &graph);
            per_graph = launches - before;   // captured, not yet run
            launches = before;
            if (st != CTR_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
            ce = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
            if (key) {
                if (cache.entries.size() >= GraphCache::CAP) {   // drop the least recently used
                    size_t lru = 0;
                    for (size_t i = 1; i < cache.entries.size(); ++i)
                        if (cache.entries[i].last_use < cache.entries[lru].last_use) lru = i;
                    cudaGraphExecDestroy(cache.entries[lru].exec);
                    cache.entries.erase(cache.entries.begin() + (long)lru);
                }
                GraphCache::Entry e;
                e.key = *key;
                e.exec = exec;
                e.per_graph = per_graph;
                e.last_use = ++cache.clock;
                cache.entries.push_back(std::move(e));
            }
        }
        for (; done + blk <= count; done += blk) {
            cudaError_t ce = cudaGraphLaunch(exec, s);
            if (ce != cudaSuccess) {
                if (!key) cudaGraphExecDestroy(exec);
                return cuda_fail(ce, "cudaGraphLaunch");
            }
            launches += per_graph;
        }
        if (!key) cudaGraphExecDestroy(exec);
    }
    for (; done < count; ++done)
        if ((st = step()) != CTR_OK) return st;
    return CTR_OK;
}

template <typename F>
ctr_status run_graphed(ctr_plan *p, int count, int blk, F &&step, cudaStream_t s,
                       const std::vector<double> *key = nullptr)
{
    return run_graphed_in(p->graphs, p->launches, count, blk, step, s, key);
}

// The plan state that decides which kernels (and shapes) the projector and FFT
// launches use, for graph keys.
// Everything a captured graph bakes in besides the launch arguments: the kernels chosen by
// the tuning hooks (group split, forward launch shape, preconditioner form) and the
// preconditioner kind.  A graph recorded under other settings is never replayed.
inline void plan_state_key(const ctr_plan *p, std::vector<double> &k)
{
    k.push_back((double)p->bp_groups);
    k.push_back((double)p->obp_groups);
    k.push_back((double)p->precond_kind);
    k.push_back((double)p->alg3);
    k.push_back((double)p->fwd_slots);
    k.push_back((double)p->fwd_segs);
    k.push_back((double)p->fft_form);
    k.push_back((double)p->pdl);
}

#ifndef CTR_POWER_GRAPH_BLOCK
#define CTR_POWER_GRAPH_BLOCK 25
#endif
constexpr int POWER_GRAPH_BLOCK = CTR_POWER_GRAPH_BLOCK;   // power-iteration steps per CUDA graph

// Power iteration for beta ~ ||R_h||: x <- R^*R x / ||R^*R x|| from the R2 start.
template <typename T>
ctr_status power_beta(ctr_plan *p, int iters, double *beta, cudaStream_t s)
{
    CTR_NVTX("power iteration beta");
    const size_t nn = (size_t)p->n * p->n;
    T *x = (T *)p->x, *xt = (T *)p->xt, *y = (T *)p->du, *g = (T *)p->gs;
    p->launches++;
    k_start_pattern<T><<<grid_for(nn), 256, 0, s>>>(x, p->n);
    ctr_status st;
    if ((st = dot2<T>(p, x, x, nn, p->d_scal, s)) != CTR_OK) return st;
    p->launches++;
    k_normalize<T><<<grid_for(nn), 256, 0, s>>>(x, nn, p->d_scal, 1, x);
    CTR_CUDA(cudaMemsetAsync(p->d_scal, 0, 2 * sizeof(double), s));
    auto step = [&]() -> ctr_status {
        ctr_status s2;
        if (fwd_needs_transpose<T>(p) && (s2 = launch_transpose<T>(p, x, xt, s)) != CTR_OK) return s2;
        if ((s2 = op_forward<T>(p, x, xt, g, 1.0, s)) != CTR_OK) return s2;
        if ((s2 = op_adjoint<T>(p, g, y, 1.0, s)) != CTR_OK) return s2;
        if ((s2 = dot2<T>(p, x, y, nn, p->d_scal, s)) != CTR_OK) return s2;
        p->launches++;
        launch_pdl(p->pdl != 0, k_normalize<T>, dim3(grid_for(nn)), dim3(256), 0, s, (const T *)y, nn,
               (const double *)p->d_scal, 1, x);
        return CTR_OK;
    };
    std::vector<double> key = {3.0, (double)POWER_GRAPH_BLOCK};
    plan_state_key(p, key);
    if ((st = run_graphed(p, iters, POWER_GRAPH_BLOCK, step, s, &key)) != CTR_OK) return st;
    CTR_CHECK_LAUNCH("power_beta");
    double h[2];
    CTR_CUDA(cudaMemcpyAsync(h, p->d_scal, sizeof(h), cudaMemcpyDeviceToHost, s));
    CTR_CUDA(cudaStreamSynchronize(s));
    if (!std::isfinite(h[0])) return fail(CTR_ENUMERIC, "power iteration for beta produced a non-finite value");
    *beta = std::sqrt(h[0] > 0 ? h[0] : 0.0);
    return CTR_OK;
}

// Power iteration for lambda_max(Mt^{-1} Rt^* Rt) in the symmetric form
// Mt^{-1/2} Rt^* Rt Mt^{-1/2}, Mt^{-1/2} = F^{-1} sqrt(||xi||_eps) F.
template <typename T>
ctr_status power_lambda(ctr_plan *p, double beta, double eps, int iters, double *lam, cudaStream_t s)
{
    CTR_NVTX("power iteration c");
    const size_t nn = (size_t)p->n * p->n;
    T *z = (T *)p->x, *x = (T *)p->u, *xt = (T *)p->xt, *yp = (T *)p->du, *y = (T *)p->t2, *g = (T *)p->gs;
    ctr_status st;
    if ((st = launch_symbols<T>(p, 1.0, 1.0, 1.0, eps, s)) != CTR_OK) return st;   // symh only matters here
    p->launches++;
    k_start_pattern<T><<<grid_for(nn), 256, 0, s>>>(z, p->n);
    if ((st = dot2<T>(p, z, z, nn, p->d_scal, s)) != CTR_OK) return st;
    p->launches++;
    k_normalize<T><<<grid_for(nn), 256, 0, s>>>(z, nn, p->d_scal, 1, z);
    CTR_CUDA(cudaMemsetAsync(p->d_scal, 0, 2 * sizeof(double), s));
    const double ib = 1.0 / beta;
    auto step = [&]() -> ctr_status {
        ctr_status s2;
        if ((s2 = launch_circulant<T>(p, z, false, (const T *)p->symh, x, 0, fwd_needs_transpose<T>(p) ? xt : nullptr,
                                      nullptr, s)) != CTR_OK)
            return s2;
        if ((s2 = op_forward<T>(p, x, xt, g, ib, s)) != CTR_OK) return s2;
        // Rt^* g; where the backprojection leaves partial images, their sum and the scale
        // run inside the preconditioner's first pass (as in the solver's step A)
        BackprojEpi<T> e{};
        e.out = yp;
        e.scale = (T)ib;
        e.outscale = T(1);
        e.inv_h = (T)(1.0 / p->h);
        const bool fuse = bp_deferred<T>(p);
        if ((s2 = launch_backproject<T>(p, g, e, s, fuse)) != CTR_OK) return s2;
        if ((s2 = launch_circulant<T>(p, yp, false, (const T *)p->symh, y, 0, nullptr, nullptr, s, nullptr, nullptr,
                                      fuse ? &e : nullptr)) != CTR_OK)
            return s2;
        if ((s2 = dot2<T>(p, z, y, nn, p->d_scal, s)) != CTR_OK) return s2;
        p->launches++;
        launch_pdl(p->pdl != 0, k_normalize<T>, dim3(grid_for(nn)), dim3(256), 0, s, (const T *)y, nn,
                   (const double *)p->d_scal, 1, z);
        return CTR_OK;
    };
    std::vector<double> key = {4.0, (double)POWER_GRAPH_BLOCK, ib};
    plan_state_key(p, key);
    if ((st = run_graphed(p, iters, POWER_GRAPH_BLOCK, step, s, &key)) != CTR_OK) return st;
    CTR_CHECK_LAUNCH("power_lambda");
    double h[2];
    CTR_CUDA(cudaMemcpyAsync(h, p->d_scal, sizeof(h), cudaMemcpyDeviceToHost, s));
    CTR_CUDA(cudaStreamSynchronize(s));
    if (!std::isfinite(h[0])) return fail(CTR_ENUMERIC, "power iteration for c produced a non-finite value");
    *lam = h[0];
    return CTR_OK;
}

template <typename T>
struct IterArgs {
    T sigma, tau, lam, inv_beta, inv_h;
    bool nonneg = false;   // Alg. 5 (u >= 0)
    bool alg3 = false;     // Alg. 3: data term in the quadratic part, only the TV term dualised
};

// One iteration of Alg. 4 (steps A-D).  diag: also keep du, t1, t2 for diagnostics.
template <typename T>
ctr_status pdrq_iteration(ctr_plan *p, const IterArgs<T> &a, bool diag, cudaStream_t s)
{
    const int n = p->n;
    const size_t nm = (size_t)p->N * p->M;
    ctr_status st;
    // A: u_tmp = -sigma (Rt^* y1 - tau div y2) into the complex FFT buffer
    BackprojEpi<T> ea{};
    ea.out = (T *)p->cbuf;
    ea.complex_out = 1;
    ea.scale = a.inv_beta;
    ea.px = (const T *)p->y2;
    ea.divtau = a.tau;
    ea.outscale = -a.sigma;
    ea.inv_h = a.inv_h;
    if (a.nonneg) {                              // Alg. 5: u_tmp = bar u - u - sigma (...)
        ea.ub = (const T *)p->ubar_u;
        ea.uu = (const T *)p->u;
    }
    const bool h = sizeof(T) == 4 && p->bf16;   // projector operands in bfloat16
    const bool fuse = bp_deferred<T>(p);        // partial-image sum and epilogue inside the first FFT pass
    if (h) {
        if constexpr (sizeof(T) == 4)
            if ((st = launch_backproject_bf16(p, p->y1h, ea, s, fuse)) != CTR_OK) return st;
    } else if ((st = launch_backproject<T>(p, (const T *)p->y1, ea, s, fuse)) != CTR_OK) {
        return st;
    }
    // B: u += F^{-1}(F(u_tmp) m), and uT (or the bfloat16 copies of u and uT)
    T *uT_out = (h || !fwd_needs_transpose<T>(p)) ? nullptr : (T *)p->uT;
    if ((st = launch_circulant<T>(p, nullptr, true, (const T *)p->sym, (T *)p->u, 1, uT_out,
                                  diag ? (T *)p->du : nullptr, s, h ? p->uh : nullptr,
                                  (h && fwd_needs_transpose<T>(p)) ? p->uTh : nullptr,
                                  fuse ? &ea : nullptr)) != CTR_OK)
        return st;
    // C: ray-driven Rt u with the data-dual step
    ForwardEpi<T> ec{};
    ec.mode = a.alg3 ? 3 : 1;
    ec.scale = a.inv_beta;
    ec.sigma = a.sigma;
    ec.Ru = (T *)p->Ru;
    ec.v1b = (T *)p->v1b;
    ec.y1 = (T *)p->y1;
    ec.t1 = diag ? (T *)p->t1 : nullptr;
    const T *d = (const T *)p->desc;
    ec.dw = d;
    ec.da = d + nm;
    ec.dlo = d + 2 * nm;
    ec.dhi = d + 3 * nm;
    const bool tv_fused = !h && sizeof(T) == 4 && p->orbit;
    const TvDualJob<T> tvj{(const T *)p->u, n, a.sigma, a.tau, a.lam, a.inv_h, (T *)p->v2b, (T *)p->y2,
                           diag ? (T *)p->t2 : nullptr, a.nonneg ? (T *)p->ubar_u : nullptr};
    if (h) {
        if constexpr (sizeof(T) == 4) {
            ec.y1h = p->y1h;
            if ((st = launch_forward_bf16(p, p->uh, p->uTh, ec, s)) != CTR_OK) return st;
        }
    } else if ((st = launch_forward<T>(p, (const T *)p->u, (const T *)p->uT, ec, s, tv_fused ? &tvj : nullptr)) !=
               CTR_OK) {
        return st;
    }
    // D: TV dual step (fused into the orbit-image kernel of step C on the FP32 symmetric path)
    if (tv_fused) return CTR_OK;
    const size_t nn = (size_t)n * n;
    p->launches++;
    k_tv_dual<T><<<grid_for(nn, 256, 4096), 256, 0, s>>>((const T *)p->u, n, a.sigma, a.tau, a.lam, a.inv_h,
                                                        (T *)p->v2b, (T *)p->y2, diag ? (T *)p->t2 : nullptr,
                                                        a.nonneg ? (T *)p->ubar_u : nullptr);
    CTR_CHECK_LAUNCH("k_tv_dual");
    return CTR_OK;
}

// Enqueue the diagnostics reductions of the current state (u, Ru, du, t1, t2) into the
// device scalars: sc[4..6] data fit / 2, max violation, data part of the gap (beta-scaled);
// sc[8..11] TV, TV part of the gap, ||du||^2, ||u||^2; sc[13] ||K^* t||^2.
template <typename T>
ctr_status enqueue_diag(ctr_plan *p, double alpha, double beta, double tau, cudaStream_t s)
{
    const int n = p->n;
    const size_t nm = (size_t)p->N * p->M, nn = (size_t)n * n;
    const T *d = (const T *)p->desc;
    const double lam = alpha / (beta * beta);
    double *sc = p->d_scal;
    int nb = grid_for(nm, RED_THREADS, p->red_blocks);
    p->launches++;
    k_diag_sino<T><<<nb, RED_THREADS, 0, s>>>((const T *)p->Ru, d, d + nm, d + 2 * nm, d + 3 * nm, (const T *)p->t1, nm, p->d_red);
    p->launches++;
    k_finalize<3><<<1, RED_THREADS, 0, s>>>(p->d_red, nb, 2u, sc + 4);
    nb = grid_for(nn, RED_THREADS, p->red_blocks);
    p->launches++;
    k_diag_img<T><<<nb, RED_THREADS, 0, s>>>((const T *)p->u, (const T *)p->du, (const T *)p->t2, n, 1.0 / p->h, lam, tau, p->d_red);
    p->launches++;
    k_finalize<4><<<1, RED_THREADS, 0, s>>>(p->d_red, nb, 0u, sc + 8);
    CTR_CHECK_LAUNCH("diagnostics");
    // dual residual K^* t = Rt^* t1 - tau div t2
    BackprojEpi<T> e{};
    e.out = (T *)p->x;
    e.complex_out = 0;
    e.scale = (T)(1.0 / beta);
    e.px = (const T *)p->t2;
    e.divtau = (T)tau;
    e.outscale = T(1);
    e.inv_h = (T)(1.0 / p->h);
    ctr_status st;
    if ((st = launch_backproject<T>(p, (const T *)p->t1, e, s)) != CTR_OK) return st;
    return dot2<T>(p, (const T *)p->x, (const T *)p->x, nn, sc + 12, s);
}

// The reported values from the device scalars of enqueue_diag (one formula for the
// host result and the device history record).
__host__ __device__ inline void diag_values(const double *h, double alpha, double beta, double c, int iters_done,
                                            bool nonneg, double *v)
{
    v[0] = beta;
    v[1] = c;
    v[3] = h[4] * beta * beta;                   // data fit
    v[4] = h[8];                                 // TV
    v[2] = v[3] + alpha * v[4];                  // objective
    v[5] = h[5] > 0 ? h[5] * beta : 0.0;         // violation
    v[6] = nonneg ? nan("") : h[6] + h[9];       // gap (Alg. 4's saddle problem only)
    v[7] = nonneg ? nan("") : sqrt(h[13]);       // dual residual
    v[8] = h[11] > 0 ? sqrt(h[10] / h[11]) : 0.0;
    v[9] = (double)iters_done;
}

__global__ void k_diag_record(const double *__restrict__ sc, double alpha, double beta, double c, int iters_done,
                              int nonneg, double *rec)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) diag_values(sc, alpha, beta, c, iters_done, nonneg != 0, rec);
}

template <typename T>
ctr_status compute_diag(ctr_plan *p, double alpha, double beta, double tau, double c, int iters_done,
                        ctr_diag *out, cudaStream_t s, bool nonneg = false)
{
    ctr_status st;
    if ((st = enqueue_diag<T>(p, alpha, beta, tau, s)) != CTR_OK) return st;
    double h[16], v[HIST_FIELDS];
    CTR_CUDA(cudaMemcpyAsync(h, p->d_scal, sizeof(h), cudaMemcpyDeviceToHost, s));
    CTR_CUDA(cudaStreamSynchronize(s));
    diag_values(h, alpha, beta, c, iters_done, nonneg, v);
    out->beta = v[0];
    out->c = v[1];
    out->objective = v[2];
    out->data_fit = v[3];
    out->tv = v[4];
    out->violation = v[5];
    out->gap = v[6];
    out->dual_residual = v[7];
    out->rel_change = v[8];
    out->iters_done = iters_done;
    if (!std::isfinite(out->objective) || !std::isfinite(out->tv))
        return fail(CTR_ENUMERIC, "non-finite objective after the solve");
    return CTR_OK;
}

// The DFT s of the impulse-response preconditioner (kind 1, Sec. "Impulse response
// preconditioners") or of the circulant one (kind 2, Sec. "Circulant matrix
// preconditioner"): the response of R_h^* R_h to the impulse at (n/2, n/2), moved to the
// origin and made point-symmetric, on the image (kind 1) or on the image flattened as
// t = i + n j (kind 2), transformed by the 2-D DFT resp. the 1-D DFT of length n^2 (real
// by the symmetry), bounded below by 1e-3 of its maximum.  Leaves it in p->pk_s.
template <typename T>
ctr_status prepare_impulse_symbol(ctr_plan *p, cudaStream_t s)
{
    const int kind = p->precond_kind;
    if (p->pk_kind == kind) return CTR_OK;
    using T2 = typename Cplx<T>::type;
    const int n = p->n, c = n / 2;
    const size_t nn = (size_t)n * n;
    T *x = (T *)p->x, *xt = (T *)p->xt, *y = (T *)p->du, *g = (T *)p->gs;
    ctr_status st;
    CTR_CUDA(cudaMemsetAsync(x, 0, nn * sizeof(T), s));
    p->launches++;
    k_set_one<T><<<1, 1, 0, s>>>(x + (size_t)c * n + c);
    CTR_CHECK_LAUNCH("k_set_one");
    if (fwd_needs_transpose<T>(p) && (st = launch_transpose<T>(p, x, xt, s)) != CTR_OK) return st;
    if ((st = op_forward<T>(p, x, xt, g, 1.0, s)) != CTR_OK) return st;
    if ((st = op_adjoint<T>(p, g, y, 1.0, s)) != CTR_OK) return st;
    p->launches++;
    k_kernel_sym<T><<<grid_for(nn, 256, 4096), 256, 0, s>>>(y, n, c, kind == 2 ? 1 : 0, xt);
    CTR_CHECK_LAUNCH("k_kernel_sym");
    if ((st = launch_fft2_forward<T>(p, xt, s, kind == 2)) != CTR_OK) return st;
    unsigned long long *mx = reinterpret_cast<unsigned long long *>(p->d_red);
    CTR_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
    p->launches += 2;
    k_real_max<T2><<<grid_for(nn, 256, 1024), 256, 0, s>>>((const T2 *)p->cbuf, nn, mx);
    k_real_floor<T, T2><<<grid_for(nn, 256, 4096), 256, 0, s>>>((const T2 *)p->cbuf, nn, mx, 1e-3, (T *)p->pk_s);
    CTR_CHECK_LAUNCH("impulse symbol");
    p->pk_kind = kind;
    return CTR_OK;
}

// ADMM with PCG inner solves (Sec. "Alternating Direction Method of Multipliers") ----
// Device scalars of the conjugate gradient: rz in two alternating slots, p.Ap in a third
// (dot2 writes two doubles per slot: the product and the second operand's square).
constexpr int CG_SLOT_RZ0 = 32, CG_SLOT_RZ1 = 34, CG_SLOT_PAP = 36;

// y = w - eta_w - Rt u (sinogram) and q = v - eta_v - grad u (image): the right-hand side
// Rt^*(w - eta_w) - tau^2 div(v - eta_v) minus A u, A = Rt^* Rt - tau^2 div grad, comes out
// of one backprojection of y with the divergence of q in its epilogue.
template <typename T>
__global__ void k_admm_resid(const T *__restrict__ w, const T *__restrict__ ew, const T *__restrict__ Ru, size_t nm,
                             const T *__restrict__ u, const T *__restrict__ v, const T *__restrict__ ev, int n,
                             T inv_h, T *y, T *q)
{
    const size_t nn = (size_t)n * n, total = nm > nn ? nm : nn;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        if (e < nm) y[e] = w[e] - ew[e] - Ru[e];
        if (e < nn) {
            T gx, gy;
            grad_at(u, n, pix_i(e, n), pix_j(e, n), inv_h, gx, gy);
            q[e] = v[e] - ev[e] - gx;
            q[e + nn] = v[e + nn] - ev[e + nn] - gy;
        }
    }
}

// alpha = rz / pAp;  u += alpha p;  r -= alpha Ap (image);  Ru += alpha Rp (sinogram)
template <typename T>
__global__ void k_cg_step(T *u, T *r, const T *__restrict__ pd, const T *__restrict__ Ap, size_t nn, T *Ru,
                          const T *__restrict__ Rp, size_t nm, const double *__restrict__ sc, int slot_rz)
{
    const T alpha = block_uniform<T>([&] {
        const double pap = sc[CG_SLOT_PAP];
        return (T)(pap != 0.0 ? sc[slot_rz] / pap : 0.0);
    });
    const size_t total = nm > nn ? nm : nn;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        if (e < nn) {
            u[e] += alpha * pd[e];
            r[e] -= alpha * Ap[e];
        }
        if (e < nm) Ru[e] += alpha * Rp[e];
    }
}

// p = z + (rz_new / rz_old) p
template <typename T>
__global__ void k_cg_dir(const T *__restrict__ z, T *pd, size_t nn, const double *__restrict__ sc, int slot_old,
                         int slot_new)
{
    const T b = block_uniform<T>([&] {
        const double old = sc[slot_old];
        return (T)(old != 0.0 ? sc[slot_new] / old : 0.0);
    });
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x)
        pd[e] = z[e] + b * pd[e];
}

// w = (ft + mu (Ru + eta_w)) / (1 + mu);  eta_w -= w - Ru;  y = w - eta_w - Ru (next right-hand side)
template <typename T>
__global__ void k_admm_sino(const T *__restrict__ Ru, const T *__restrict__ ft, T *w, T *ew, size_t nm, T mu,
                            T *y)
{
    const T inv = T(1) / (T(1) + mu);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nm; e += (size_t)gridDim.x * blockDim.x) {
        const T ru = Ru[e];
        const T wn = (ft[e] + mu * (ru + ew[e])) * inv;
        const T en = ew[e] - (wn - ru);
        w[e] = wn;
        ew[e] = en;
        y[e] = wn - en - ru;
    }
}

// g = grad u;  v = shrink(g + eta_v, thr);  eta_v -= v - g;  q = v - eta_v - g
template <typename T>
__global__ void k_admm_img(const T *__restrict__ u, int n, T inv_h, T thr, T *v, T *ev, T *q)
{
    const size_t nn = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        T gx, gy;
        grad_at(u, n, pix_i(e, n), pix_j(e, n), inv_h, gx, gy);
        const T ax = gx + ev[e], ay = gy + ev[e + nn];
        const T nrm = sqrt(ax * ax + ay * ay);
        const T fac = nrm > thr ? T(1) - thr / nrm : T(0);
        const T vx = fac * ax, vy = fac * ay;
        const T ex = ev[e] - (vx - gx), ey = ev[e + nn] - (vy - gy);
        v[e] = vx;
        v[e + nn] = vy;
        ev[e] = ex;
        ev[e + nn] = ey;
        q[e] = vx - ex - gx;
        q[e + nn] = vy - ey - gy;
    }
}

// Dual certificates of the saddle problem for the diagnostics: t1 = Rt u - ft,
// t2 = mu tau eta_v; du = u - u_prev.
template <typename T>
__global__ void k_admm_diag(const T *__restrict__ Ru, const T *__restrict__ ft, size_t nm, const T *__restrict__ ev,
                            const T *__restrict__ u, const T *__restrict__ uprev, size_t nn, T mutau, T *t1, T *t2,
                            T *du)
{
    const size_t total = nm > 2 * nn ? nm : 2 * nn;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        if (e < nm) t1[e] = Ru[e] - ft[e];
        if (e < 2 * nn) t2[e] = mutau * ev[e];
        if (e < nn) du[e] = u[e] - uprev[e];
    }
}

// One ADMM iteration.  Buffers: u = p->u, Rt u = p->Ru (kept up to date through the CG
// updates, Rt(u + alpha p) = Rt u + alpha Rt p), w = p->v1b, eta_w = p->y1, v = p->v2b,
// eta_v = p->y2; y (sinogram) in p->gs and q (image pair) in p->t2 on entry; CG
// scratch: r = p->du, z = p->x, p = p->ubar_u, A p = p->xt, grad p = p->t2, Rt p = p->gs.
template <typename T>
ctr_status admm_iteration(ctr_plan *p, int cg_iters, T tau, T mu, T lam, T inv_beta, cudaStream_t s)
{
    const int n = p->n;
    const size_t nn = (size_t)n * n, nm = (size_t)p->N * p->M;
    const T inv_h = (T)(1.0 / p->h), tau2 = tau * tau;
    T *u = (T *)p->u, *Ru = (T *)p->Ru, *r = (T *)p->du, *z = (T *)p->x, *pd = (T *)p->ubar_u, *Ap = (T *)p->xt;
    T *gs = (T *)p->gs, *t2 = (T *)p->t2;
    double *sc = p->d_scal;
    ctr_status st;
    BackprojEpi<T> eb{};
    eb.complex_out = 0;
    eb.scale = inv_beta;
    eb.px = t2;
    eb.divtau = tau2;
    eb.outscale = T(1);
    eb.inv_h = inv_h;
    // r = b - A u;  z = M^{-1} r (p = z as a second output);  rz = r.z
    eb.out = r;
    if ((st = launch_backproject<T>(p, gs, eb, s)) != CTR_OK) return st;
    if ((st = launch_circulant<T>(p, r, false, (const T *)p->sym, z, 0, nullptr, pd, s)) != CTR_OK) return st;
    if ((st = dot2<T>(p, r, z, nn, sc + CG_SLOT_RZ0, s)) != CTR_OK) return st;
    for (int k = 0; k < cg_iters; ++k) {
        const int so = (k & 1) ? CG_SLOT_RZ1 : CG_SLOT_RZ0, sn = (k & 1) ? CG_SLOT_RZ0 : CG_SLOT_RZ1;
        if (fwd_needs_transpose<T>(p) && (st = launch_transpose<T>(p, pd, (T *)p->uT, s)) != CTR_OK) return st;
        if ((st = op_forward<T>(p, pd, (const T *)p->uT, gs, (double)inv_beta, s)) != CTR_OK) return st;
        if ((st = op_grad<T>(p, pd, t2, s)) != CTR_OK) return st;
        eb.out = Ap;
        if ((st = launch_backproject<T>(p, gs, eb, s)) != CTR_OK) return st;
        if ((st = dot2<T>(p, pd, Ap, nn, sc + CG_SLOT_PAP, s)) != CTR_OK) return st;
        p->launches++;
        k_cg_step<T><<<grid_for(nm > nn ? nm : nn, 256, 4096), 256, 0, s>>>(u, r, pd, Ap, nn, Ru, gs, nm, sc, so);
        CTR_CHECK_LAUNCH("k_cg_step");
        if (k + 1 == cg_iters) break;   // the last direction would not be used
        if ((st = launch_circulant<T>(p, r, false, (const T *)p->sym, z, 0, nullptr, nullptr, s)) != CTR_OK) return st;
        if ((st = dot2<T>(p, r, z, nn, sc + sn, s)) != CTR_OK) return st;
        p->launches++;
        k_cg_dir<T><<<grid_for(nn, 256, 4096), 256, 0, s>>>(z, pd, nn, sc, so, sn);
        CTR_CHECK_LAUNCH("k_cg_dir");
    }
    p->launches += 2;
    k_admm_sino<T><<<grid_for(nm, 256, 4096), 256, 0, s>>>(Ru, (const T *)p->desc + nm, (T *)p->v1b, (T *)p->y1, nm,
                                                          mu, gs);
    k_admm_img<T><<<grid_for(nn, 256, 4096), 256, 0, s>>>(u, n, inv_h, lam / (mu * tau2), (T *)p->v2b, (T *)p->y2,
                                                         t2);
    CTR_CHECK_LAUNCH("admm updates");
    return CTR_OK;
}

// ADMM from zero on the beta-scaled unconstrained problem; desc holds (1, ft, -inf, +inf).
template <typename T>
ctr_status admm_loop(ctr_plan *p, double alpha, int iters, int cg_iters, double mu, const ctr_params &prm,
                     double beta, double c, ctr_diag *diag, cudaStream_t s)
{
    const int n = p->n;
    const size_t nn = (size_t)n * n, nm = (size_t)p->N * p->M;
    ctr_status st;
    // PCG preconditioner for Rt^* Rt + tau^2 (-Delta_h): M = c S + tau^2 Lap (sigma = 1)
    if ((st = launch_symbols<T>(p, 1.0, prm.tau, c, prm.eps, s, false)) != CTR_OK) return st;
    CTR_CUDA(cudaMemsetAsync(p->u, 0, nn * sizeof(T), s));
    CTR_CUDA(cudaMemsetAsync(p->Ru, 0, nm * sizeof(T), s));
    CTR_CUDA(cudaMemsetAsync(p->v1b, 0, nm * sizeof(T), s));
    CTR_CUDA(cudaMemsetAsync(p->y1, 0, nm * sizeof(T), s));
    CTR_CUDA(cudaMemsetAsync(p->v2b, 0, 2 * nn * sizeof(T), s));
    CTR_CUDA(cudaMemsetAsync(p->y2, 0, 2 * nn * sizeof(T), s));
    p->launches++;
    k_admm_resid<T><<<grid_for(nm > nn ? nm : nn, 256, 4096), 256, 0, s>>>(
        (const T *)p->v1b, (const T *)p->y1, (const T *)p->Ru, nm, (const T *)p->u, (const T *)p->v2b,
        (const T *)p->y2, n, (T)(1.0 / p->h), (T *)p->gs, (T *)p->t2);
    CTR_CHECK_LAUNCH("k_admm_resid");
    const T tau = (T)prm.tau, mu_t = (T)mu, lam = (T)(alpha / (beta * beta)), inv_beta = (T)(1.0 / beta);
    auto one = [&]() { return admm_iteration<T>(p, cg_iters, tau, mu_t, lam, inv_beta, s); };
    const int body = iters > 0 ? iters - 1 : 0;
    std::vector<double> key = {5.0, (double)prm.graph_block, (double)cg_iters, (double)tau, (double)mu_t, (double)lam,
                               (double)inv_beta};
    plan_state_key(p, key);
    p->hist_count = 0;
    if ((st = run_graphed(p, body, prm.graph_block, one, s, &key)) != CTR_OK) return st;
    if (iters > 0) {
        CTR_CUDA(cudaMemcpyAsync(p->aux, p->u, nn * sizeof(T), cudaMemcpyDeviceToDevice, s));
        if ((st = one()) != CTR_OK) return st;
    } else {
        CTR_CUDA(cudaMemsetAsync(p->aux, 0, nn * sizeof(T), s));
    }
    if (!diag) return CTR_OK;
    p->launches++;
    k_admm_diag<T><<<grid_for(nm > 2 * nn ? nm : 2 * nn, 256, 4096), 256, 0, s>>>(
        (const T *)p->Ru, (const T *)p->desc + nm, nm, (const T *)p->y2, (const T *)p->u, (const T *)p->aux, nn,
        (T)(mu * prm.tau), (T *)p->t1, (T *)p->t2, (T *)p->du);
    CTR_CHECK_LAUNCH("k_admm_diag");
    return compute_diag<T>(p, alpha, beta, prm.tau, c, iters, diag, s);
}

// Metal-trace estimation (Sec. "Real metal artifacts"): the pixels whose value exceeds
// the threshold, dilated by the disk {di^2 + dj^2 <= r^2}, as a 0/1 image (in the
// projector's operand type) and optionally as bytes.  Comparisons in FP64, so that the
// decision does not depend on the image's storage type.
template <typename T, typename S>
__global__ void k_mark_dilate(const T *__restrict__ u, int n, double thr, int r, uint8_t *marked, S *img)
{
    const size_t nn = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const int i = pix_i(e, n), j = pix_j(e, n);
        bool hit = false;
        for (int di = -r; di <= r && !hit; ++di) {
            const int ii = i + di;
            if (ii < 0 || ii >= n) continue;
            int w = r;
            while (w * w + di * di > r * r) --w;
            const int j0 = max(j - w, 0), j1 = min(j + w, n - 1);
            for (int jj = j0; jj <= j1; ++jj)
                if ((double)u[(size_t)ii * n + jj] > thr) {
                    hit = true;
                    break;
                }
        }
        if (marked) marked[e] = hit ? 1 : 0;
        img[e] = hit ? S(1.0f) : S(0.0f);
    }
}

template <typename T>
__global__ void k_trace_from_sino(const T *__restrict__ g, size_t len, double tol, uint8_t *trace)
{
    for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < len; r += (size_t)gridDim.x * blockDim.x)
        trace[r] = (double)g[r] > tol ? 1 : 0;
}

// marks -> R_h of the 0/1 image -> bins above proj_tol.  Scratch: x, uT (or the bfloat16
// operand copies), gs.
template <typename T>
ctr_status metal_trace(ctr_plan *p, const T *u, double thr, int radius, double proj_tol, uint8_t *marked,
                       uint8_t *trace, cudaStream_t s)
{
    const int n = p->n;
    const size_t nn = (size_t)n * n, nm = (size_t)p->N * p->M;
    T *g = (T *)p->gs;
    ctr_status st;
    p->launches++;
    if constexpr (sizeof(T) == 4) {
        if (p->bf16) {
            k_mark_dilate<T, __nv_bfloat16><<<grid_for(nn, 256, 4096), 256, 0, s>>>(u, n, thr, radius, marked, p->uh);
            CTR_CHECK_LAUNCH("k_mark_dilate");
            if (fwd_needs_transpose<float>(p) && (st = launch_transpose<__nv_bfloat16>(p, p->uh, p->uTh, s)) != CTR_OK)
                return st;
            if ((st = op_forward_bf16(p, p->uh, p->uTh, (float *)g, s)) != CTR_OK) return st;
            p->launches++;
            k_trace_from_sino<float><<<grid_for(nm, 256, 4096), 256, 0, s>>>((const float *)g, nm, proj_tol, trace);
            CTR_CHECK_LAUNCH("k_trace_from_sino");
            return CTR_OK;
        }
    }
    T *x = (T *)p->x;
    k_mark_dilate<T, T><<<grid_for(nn, 256, 4096), 256, 0, s>>>(u, n, thr, radius, marked, x);
    CTR_CHECK_LAUNCH("k_mark_dilate");
    if (fwd_needs_transpose<T>(p) && (st = launch_transpose<T>(p, x, (T *)p->uT, s)) != CTR_OK) return st;
    if ((st = op_forward<T>(p, x, (const T *)p->uT, g, 1.0, s)) != CTR_OK) return st;
    p->launches++;
    k_trace_from_sino<T><<<grid_for(nm, 256, 4096), 256, 0, s>>>(g, nm, proj_tol, trace);
    CTR_CHECK_LAUNCH("k_trace_from_sino");
    return CTR_OK;
}

// Alg. 1 (Chambolle-Pock) on the beta-scaled (C_h), from zero: the unpreconditioned
// baseline.  State: u (p->u), u_bar (p->ubar_u), v (p->v1b), w (p->v2b).  One iteration:
//   v = prox_{tau g*}(v + tau Rt u_bar)          forward projection of u_bar + epilogue (mode 2)
//   w = P_lambda(w + tau grad u_bar)             k_cp_tv
//   u_new = u + sigma div w - sigma Rt^* v,  u_bar = 2 u_new - u   backprojection + epilogue
// sp = sigma (primal step), sd = tau (dual step) in the notation of Alg. 1.  tau4 is the
// tau of Alg. 4's saddle form used to report the diagnostics (t2 = w / tau4).
template <typename T>
ctr_status cp_loop(ctr_plan *p, double alpha, int iters, const ctr_params &prm, double beta, double sp, double sd,
                   ctr_diag *diag, cudaStream_t s)
{
    const int n = p->n;
    const size_t nn = (size_t)n * n, nm = (size_t)p->N * p->M;
    const T lam = (T)(alpha / (beta * beta)), inv_h = (T)(1.0 / p->h);
    T *u = (T *)p->u, *ub = (T *)p->ubar_u, *v = (T *)p->v1b, *w = (T *)p->v2b;
    const T *d = (const T *)p->desc;
    CTR_CUDA(cudaMemsetAsync(u, 0, nn * sizeof(T), s));
    CTR_CUDA(cudaMemsetAsync(ub, 0, nn * sizeof(T), s));
    CTR_CUDA(cudaMemsetAsync(v, 0, nm * sizeof(T), s));
    CTR_CUDA(cudaMemsetAsync(w, 0, 2 * nn * sizeof(T), s));
    auto one = [&]() -> ctr_status {
        ctr_status st;
        ForwardEpi<T> ec{};
        ec.mode = 2;
        ec.scale = (T)(1.0 / beta);
        ec.sigma = (T)sd;
        ec.v1b = v;
        ec.dw = d;
        ec.da = d + nm;
        ec.dlo = d + 2 * nm;
        ec.dhi = d + 3 * nm;
        if (fwd_needs_transpose<T>(p) && (st = launch_transpose<T>(p, ub, (T *)p->uT, s)) != CTR_OK) return st;
        if ((st = launch_forward<T>(p, ub, (const T *)p->uT, ec, s)) != CTR_OK) return st;
        p->launches++;
        k_cp_tv<T><<<grid_for(nn, 256, 4096), 256, 0, s>>>(ub, n, (T)sd, lam, inv_h, w);
        CTR_CHECK_LAUNCH("k_cp_tv");
        BackprojEpi<T> eb{};
        eb.out = u;
        eb.scale = (T)(1.0 / beta);
        eb.px = w;
        eb.divtau = T(1);
        eb.outscale = (T)(-sp);
        eb.inv_h = inv_h;
        eb.ub = u;              // + u (old)
        eb.bar_out = ub;        // u_bar = 2 u_new - u
        return launch_backproject<T>(p, v, eb, s);
    };
    ctr_status st;
    const int blk = prm.graph_block > 0 ? prm.graph_block : 0;
    std::vector<double> key = {2.0, (double)blk, (double)lam, sp, sd, beta, (double)inv_h};
    plan_state_key(p, key);
    p->hist_count = 0;
    if ((st = run_graphed(p, iters, blk, one, s, &key)) != CTR_OK) return st;
    if (!diag) return CTR_OK;
    // diagnostics of the saddle problem of Alg. 4 at (u; t1 = v, t2 = w / tau4); du = u - u_prev
    const T tau4 = (T)prm.tau;
    p->launches += 3;
    k_axpy<T><<<grid_for(nn, 256, 4096), 256, 0, s>>>(ub, u, T(-1), nn, (T *)p->du);   // u_bar - u = u - u_prev
    k_axpy<T><<<grid_for(nm, 256, 4096), 256, 0, s>>>(v, v, T(0), nm, (T *)p->t1);
    k_axpy<T><<<grid_for(2 * nn, 256, 4096), 256, 0, s>>>(w, w, T(1) / tau4 - T(1), 2 * nn, (T *)p->t2);
    CTR_CHECK_LAUNCH("cp diagnostics set-up");
    if (fwd_needs_transpose<T>(p) && (st = launch_transpose<T>(p, u, (T *)p->uT, s)) != CTR_OK) return st;
    if ((st = op_forward<T>(p, u, (const T *)p->uT, (T *)p->Ru, 1.0 / beta, s)) != CTR_OK) return st;
    return compute_diag<T>(p, alpha, beta, prm.tau, 0.0, iters, diag, s);
}

// Full solve on the plan's internal stream.  desc must already hold the
// beta-scaled data term; u, Ru, v1b, v2b hold the start state.
template <typename T>
ctr_status pdrq_loop(ctr_plan *p, double alpha, int iters, const ctr_params &prm, double beta, double c,
                     ctr_diag *diag, cudaStream_t s)
{
    CTR_NVTX("iterations");
    const int n = p->n;
    const size_t nn = (size_t)n * n, nm = (size_t)p->N * p->M;
    IterArgs<T> a;
    a.sigma = (T)prm.sigma;
    a.tau = (T)prm.tau;
    a.lam = (T)(alpha / (beta * beta));
    a.inv_beta = (T)(1.0 / beta);
    a.inv_h = (T)(1.0 / p->h);
    a.nonneg = prm.nonneg != 0;
    a.alg3 = p->alg3;
    ctr_status st;
    // Alg. 3's M carries sigma c where Alg. 4's carries sigma^2 c
    const double c_sym = a.alg3 ? c / prm.sigma : c;
    if ((st = launch_symbols<T>(p, prm.sigma, prm.tau, c_sym, prm.eps, s, a.nonneg)) != CTR_OK) return st;
    // y1 = v1b + sigma Ru (Alg. 3: the residual Ru - ft) ; y2 = v2b + sigma tau grad u
    p->launches++;
    if (a.alg3)
        k_axpy<T><<<grid_for(nm, 256, 4096), 256, 0, s>>>((const T *)p->Ru, (const T *)p->desc + nm, T(-1), nm,
                                                          (T *)p->y1);
    else
        k_axpy<T><<<grid_for(nm, 256, 4096), 256, 0, s>>>((const T *)p->v1b, (const T *)p->Ru, a.sigma, nm,
                                                          (T *)p->y1);
    p->launches++;
    k_init_y2<T><<<grid_for(nn, 256, 4096), 256, 0, s>>>((const T *)p->u, (const T *)p->v2b, n, a.sigma * a.tau, a.inv_h, (T *)p->y2);
    if (sizeof(T) == 4 && p->bf16) {
        p->launches++;
        k_to_bf16<<<grid_for(nm, 256, 4096), 256, 0, s>>>((const float *)p->y1, nm, p->y1h);
    }
    CTR_CHECK_LAUNCH("pdrq init");
    if (iters <= 0) {
        CTR_CUDA(cudaMemsetAsync(p->du, 0, nn * sizeof(T), s));
        CTR_CUDA(cudaMemsetAsync(p->t1, 0, nm * sizeof(T), s));
        CTR_CUDA(cudaMemsetAsync(p->t2, 0, 2 * nn * sizeof(T), s));
        p->hist_count = 0;
        if (diag) return compute_diag<T>(p, alpha, beta, prm.tau, c, 0, diag, s, a.nonneg);
        return CTR_OK;
    }
    // graphs of plain iterations, reused across calls while the key holds
    const int blk = prm.graph_block > 0 ? prm.graph_block : 0;
    std::vector<double> key = {1.0, (double)blk, (double)a.sigma, (double)a.tau, (double)a.lam, (double)a.inv_beta,
                               (double)a.inv_h, (double)a.nonneg};
    plan_state_key(p, key);
    auto plain = [&]() { return pdrq_iteration<T>(p, a, false, s); };
    p->hist_count = 0;
    int done = 0;
    bool stopped = false;
    const int ce = prm.check_every;
    if (ce > 0) {
        // a check after every ce iterations: the last iteration of each segment keeps du,
        // t1, t2, the reductions and one record stay on the device (no host round trip
        // unless stop_tol asks for rel_change)
        while (iters - done >= ce) {
            if ((st = run_graphed(p, ce - 1, blk, plain, s, &key)) != CTR_OK) return st;
            if ((st = pdrq_iteration<T>(p, a, true, s)) != CTR_OK) return st;
            done += ce;
            if (p->hist_count >= MAX_CHECKS) return fail(CTR_EINVAL, "more diagnostics checks than the plan holds");
            if ((st = enqueue_diag<T>(p, alpha, beta, prm.tau, s)) != CTR_OK) return st;
            double *rec = p->d_hist + (size_t)p->hist_count * HIST_FIELDS;
            p->launches++;
            k_diag_record<<<1, 32, 0, s>>>(p->d_scal, alpha, beta, c, done, a.nonneg ? 1 : 0, rec);
            CTR_CHECK_LAUNCH("k_diag_record");
            ++p->hist_count;
            if (prm.stop_tol > 0) {
                double rel = 0;
                CTR_CUDA(cudaMemcpyAsync(&rel, rec + 8, sizeof(double), cudaMemcpyDeviceToHost, s));
                CTR_CUDA(cudaStreamSynchronize(s));
                if (rel <= prm.stop_tol) {
                    stopped = true;
                    break;
                }
            }
            if (done == iters) break;
        }
    }
    if (!stopped && done < iters) {   // the rest; the last iteration also keeps du, t1, t2
        if ((st = run_graphed(p, iters - done - 1, blk, plain, s, &key)) != CTR_OK) return st;
        if ((st = pdrq_iteration<T>(p, a, true, s)) != CTR_OK) return st;
        done = iters;
    }
    if (diag) return compute_diag<T>(p, alpha, beta, prm.tau, c, done, diag, s, a.nonneg);
    return CTR_OK;
}

template <typename T>
ctr_status build_desc_from_data(ctr_plan *p, const T *f, const uint8_t *mask, double delta, double ratio, double beta,
                                cudaStream_t s)
{
    const size_t nm = (size_t)p->N * p->M;
    T *d = (T *)p->desc;
    p->launches++;
    k_make_desc<T><<<grid_for(nm, 256, 4096), 256, 0, s>>>(f, mask, nm, delta, ratio, 1.0 / beta, d, d + nm, d + 2 * nm, d + 3 * nm);
    CTR_CHECK_LAUNCH("k_make_desc");
    return CTR_OK;
}

template <typename T>
ctr_status build_desc_from_arrays(ctr_plan *p, const T *w, const T *a, const T *lo, const T *hi, double beta, cudaStream_t s)
{
    const size_t nm = (size_t)p->N * p->M;
    T *d = (T *)p->desc;
    p->launches++;
    k_scale_desc<T><<<grid_for(nm, 256, 4096), 256, 0, s>>>(w, a, lo, hi, nm, 1.0 / beta, d, d + nm, d + 2 * nm, d + 3 * nm);
    CTR_CHECK_LAUNCH("k_scale_desc");
    return CTR_OK;
}

// ------------------------------------------------------------------------------
// Reverse mode of one iteration of Alg. 4 (hand-written vector-Jacobian product).
// The iteration maps s_k = (u, v1b, v2b) to s_{k+1}; with Ru = Rt u,
//   u'   = u - sigma P( Rt^*(v1b + sigma Rt u) - tau div(v2b + sigma tau grad u) )
//   z1   = v1b + 2 sigma Rt u',  t1 = z1 - sigma clip((z1 + w a)/(sigma + w), lo, hi)
//   v1b' = t1 - sigma Rt u'
//   z2   = v2b + 2 sigma tau grad u',  t2 = z2 / max(1, tau |z2| / lam)
//   v2b' = t2 - sigma tau grad u'
// Given cotangents (bu, b1, b2) of (u', v1b', v2b') it returns those of (u, v1b,
// v2b) in place and accumulates the cotangents of the data f (through a, lo, hi)
// and of alpha (through lam = alpha/beta^2).  z1, z2 are recomputed from s_k and
// s_{k+1}.  Kinks of clip and of the projection take the inside branch.
// ------------------------------------------------------------------------------
namespace {

template <typename T>
__global__ void k_vjp_data(const T *__restrict__ v1b0, const T *__restrict__ Ru1, const T *__restrict__ f,
                           const uint8_t *__restrict__ mask, size_t len, double delta, double ratio, double inv_beta,
                           T sigma, T *b1, T *dRu, T *gf)
{
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < len; r += (size_t)gridDim.x * blockDim.x) {
        // the beta-scaled data term exactly as k_make_desc builds it
        const double fv = (double)f[r];
        const bool tr = mask && mask[r];
        const T w = tr ? T(0) : T(1);
        const T a = tr ? T(0) : (T)(fv * inv_beta);
        const T lo = tr ? (T)(ratio * fv * inv_beta) : (T)(delta >= 0 ? (fv - delta) * inv_beta : -inf);
        const T hi = tr ? (T)inf : (T)(delta >= 0 ? (fv + delta) * inv_beta : inf);
        const T z1 = v1b0[r] + T(2) * sigma * Ru1[r];
        const T q = (z1 + w * a) / (sigma + w);
        const bool below = q < lo, above = q > hi, in = !below && !above;
        const T A1 = b1[r];
        const T dz1 = in ? A1 * (T(1) - sigma / (sigma + w)) : A1;
        const T da = in ? -sigma * w / (sigma + w) * A1 : T(0);
        const T dlo = below ? -sigma * A1 : T(0);
        const T dhi = above ? -sigma * A1 : T(0);
        // d(a, lo, hi)/df: off the trace 1/beta each (lo, hi only when bounded); on it ratio/beta for lo
        const T ib = (T)inv_beta;
        gf[r] += tr ? (T)ratio * ib * dlo : ib * (da + dlo + dhi);
        dRu[r] = -sigma * A1 + T(2) * sigma * dz1;
        b1[r] = dz1;
    }
}

template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
k_vjp_tv(const T *__restrict__ u1, const T *__restrict__ v2b0, int n, T sigma, T tau, T lam, T inv_h, T *b2, T *dg,
         double *part)
{
    const size_t nn = (size_t)n * n;
    const T st = sigma * tau;
    double v[1] = {0.0};
    for (size_t e = blockIdx.x * (size_t)RED_THREADS + threadIdx.x; e < nn; e += (size_t)gridDim.x * RED_THREADS) {
        T gx, gy;
        grad_at(u1, n, pix_i(e, n), pix_j(e, n), inv_h, gx, gy);
        const T zx = v2b0[e] + T(2) * st * gx, zy = v2b0[e + nn] + T(2) * st * gy;
        const T ax = b2[e], ay = b2[e + nn];
        const T nz = sqrt(zx * zx + zy * zy);
        T dx = ax, dy = ay;
        if (tau * nz > lam) {            // projected: t2 = (lam/tau) z/|z|
            const T nx = zx / nz, ny = zy / nz;
            const T dot = nx * ax + ny * ay;
            const T s = lam / (tau * nz);
            dx = s * (ax - nx * dot);
            dy = s * (ay - ny * dot);
            v[0] += (double)dot / (double)tau;     // d t2 / d lam = z / (tau |z|)
        }
        b2[e] = dx;
        b2[e + nn] = dy;
        dg[e] = -st * ax + T(2) * st * dx;
        dg[e + nn] = -st * ay + T(2) * st * dy;
    }
    block_reduce<1>(v, 0u, part + blockIdx.x);
}

__global__ void k_accum_scalar(const double *__restrict__ src, double scale, double *dst)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst += scale * *src;
}

template <typename T>
__global__ void k_scal(const T *__restrict__ x, T s, size_t len, T *y)
{
    for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < len; r += (size_t)gridDim.x * blockDim.x)
        y[r] = s * x[r];
}

}  // namespace

template <typename T>
ctr_status pdrq_vjp_step(ctr_plan *p, const T *u0, const T *v1b0, const T *v2b0, const T *u1, const T *Ru1,
                         const T *f, const uint8_t *mask, double delta, double ratio, double alpha, double beta,
                         double c, const ctr_params &prm, T *bu, T *b1, T *b2, T *gf, double *galpha, cudaStream_t s)
{
    (void)u0;
    const int n = p->n;
    const size_t nn = (size_t)n * n, nm = (size_t)p->N * p->M;
    const T sigma = (T)prm.sigma, tau = (T)prm.tau, inv_h = (T)(1.0 / p->h);
    const double ib = 1.0 / beta;
    const T lam = (T)(alpha * ib * ib);
    T *dRu = (T *)p->gs;            // sinogram scratch
    T *dy1 = (T *)p->t1;            // sinogram scratch
    T *dg = (T *)p->y2;             // 2 n^2
    T *dy2 = (T *)p->t2;            // 2 n^2
    T *du1 = (T *)p->du;            // n^2
    T *dr = (T *)p->x;              // n^2
    T *drT = (T *)p->xt;            // n^2
    ctr_status st;
    if ((st = launch_symbols<T>(p, prm.sigma, prm.tau, c, prm.eps, s)) != CTR_OK) return st;
    // data and TV pointwise steps
    p->launches += 4;
    k_vjp_data<T><<<grid_for(nm, 256, 4096), 256, 0, s>>>(v1b0, Ru1, f, mask, nm, delta, ratio, ib, sigma, b1, dRu, gf);
    const int nb = grid_for(nn, RED_THREADS, p->red_blocks);
    k_vjp_tv<T><<<nb, RED_THREADS, 0, s>>>(u1, v2b0, n, sigma, tau, lam, inv_h, b2, dg, p->d_red);
    k_finalize<1><<<1, RED_THREADS, 0, s>>>(p->d_red, nb, 0u, p->d_scal + 20);
    k_accum_scalar<<<1, 32, 0, s>>>(p->d_scal + 20, ib * ib, galpha);
    CTR_CHECK_LAUNCH("vjp pointwise");
    // du' = bu + Rt^* dRu - div(dg)   (bu added in the backprojection's epilogue)
    BackprojEpi<T> e{};
    e.out = du1;
    e.scale = (T)ib;
    e.px = dg;
    e.divtau = T(1);
    e.outscale = T(1);
    e.inv_h = inv_h;
    e.ub = bu;
    if ((st = launch_backproject<T>(p, dRu, e, s)) != CTR_OK) return st;
    // dr = -sigma P(du'): P(du') is kept unscaled and -sigma goes into the two consumers
    const bool tr = fwd_needs_transpose<T>(p);
    if ((st = launch_circulant<T>(p, du1, false, (const T *)p->sym, dr, 0, tr ? drT : nullptr, nullptr, s)) != CTR_OK)
        return st;
    // dy1 = Rt dr = -sigma Rt P(du') ; dy2 = tau grad dr = -sigma tau grad P(du')
    if ((st = op_forward<T>(p, dr, drT, dy1, -prm.sigma * ib, s)) != CTR_OK) return st;
    if ((st = op_grad<T>(p, dr, dy2, s)) != CTR_OK) return st;
    p->launches += 1;
    k_scal<T><<<grid_for(2 * nn, 256, 4096), 256, 0, s>>>(dy2, -sigma * tau, 2 * nn, dy2);
    // du = du' + sigma Rt^* dy1 - sigma tau div(dy2)   (du' added in the epilogue, into bu)
    BackprojEpi<T> e2{};
    e2.out = bu;
    e2.scale = (T)(prm.sigma * ib);
    e2.px = dy2;
    e2.divtau = sigma * tau;
    e2.outscale = T(1);
    e2.inv_h = inv_h;
    e2.ub = du1;
    if ((st = launch_backproject<T>(p, dy1, e2, s)) != CTR_OK) return st;
    p->launches += 2;
    // dv1b = dz1 + dy1 ; dv2b = dz2 + dy2
    k_axpy<T><<<grid_for(nm, 256, 4096), 256, 0, s>>>(b1, dy1, T(1), nm, b1);
    k_axpy<T><<<grid_for(2 * nn, 256, 4096), 256, 0, s>>>(b2, dy2, T(1), 2 * nn, b2);
    CTR_CHECK_LAUNCH("vjp step");
    return CTR_OK;
}

template ctr_status pdrq_vjp_step<float>(ctr_plan *, const float *, const float *, const float *, const float *,
                                         const float *, const float *, const uint8_t *, double, double, double, double,
                                         double, const ctr_params &, float *, float *, float *, float *, double *,
                                         cudaStream_t);
template ctr_status pdrq_vjp_step<double>(ctr_plan *, const double *, const double *, const double *, const double *,
                                          const double *, const double *, const uint8_t *, double, double, double,
                                          double, double, const ctr_params &, double *, double *, double *, double *,
                                          double *, cudaStream_t);

ctr_status launch_batch_tv(const SliceDesc *sd, const int *prefix, int ns, int blocks, cudaStream_t s)
{
    if (blocks <= 0) return CTR_OK;
    k_tv_dual_batch<<<blocks, 256, 0, s>>>(sd, prefix, ns);
    CTR_CHECK_LAUNCH("k_tv_dual_batch");
    return CTR_OK;
}

// ------------------------------------------------------------------------------
// Batched solve: per-slice set-up (power iterations, data term, start state,
// symbols) on the batch stream, then iterations 1..iters-1 with one launch per
// stage over all slices (captured as CUDA graphs of graph_block iterations), and the
// last iteration per slice so that each slice keeps the dual certificates for its
// diagnostics.
// ------------------------------------------------------------------------------
bool batch_slice_packed(const ctr_batch *b, const ctr_plan *p);
ctr_status batch_prepare(ctr_batch *b);

ctr_status batch_solve(ctr_batch *b, const float *const *f, const uint8_t *const *mask, const double *alpha,
                       const double *delta, int iters, const ctr_params &prm, const double *betas, const double *cs,
                       float *const *u_out, ctr_diag *diags, cudaStream_t s)
{
    const int ns = (int)b->plans.size();
    // the circulant preconditioner's twisted column pass needs the complex form: the stage
    // tables follow the kind of this solve
    const int packed = prm.precond == 2 ? 0 : 1;
    if (b->fft_packed != packed) {
        b->fft_packed = packed;
        ctr_status sp = batch_prepare(b);
        if (sp != CTR_OK) return sp;
    }
    std::vector<SliceDesc> hd(ns);
    std::vector<IterArgs<float>> args(ns);
    std::vector<double> beta(ns), c(ns);
    ctr_status st;
    for (int i = 0; i < ns; ++i) {
        ctr_plan *p = b->plans[i];
        const unsigned long long l0 = p->launches;
        p->precond_kind = prm.precond;                 // the preconditioner kind (its kernel built once per plan)
        if ((prm.precond == 1 || prm.precond == 2) && (st = prepare_impulse_symbol<float>(p, s)) != CTR_OK) return st;
        beta[i] = betas ? betas[i] : 0.0;
        if (!(beta[i] > 0)) {
            if ((st = power_beta<float>(p, prm.power_iters, &beta[i], s)) != CTR_OK) return st;
            if (!(beta[i] > 0)) return fail(CTR_ENUMERIC, "power iteration gave ||R_h|| = 0");
        }
        const double eps = prm.eps > 0 ? prm.eps : 3.14159265358979323846 / p->n;
        c[i] = cs ? cs[i] : 0.0;
        if (!(c[i] > 0)) {
            double lam = 0;
            if ((st = power_lambda<float>(p, beta[i], eps, prm.power_iters, &lam, s)) != CTR_OK) return st;
            c[i] = prm.c_margin * lam;
        }
        if ((st = build_desc_from_data<float>(p, f[i], mask ? mask[i] : nullptr, delta[i], prm.trace_ratio, beta[i], s)) != CTR_OK)
            return st;
        const size_t nn = (size_t)p->n * p->n, nm = (size_t)p->N * p->M;
        CTR_CUDA(cudaMemsetAsync(p->u, 0, nn * sizeof(float), s));
        CTR_CUDA(cudaMemsetAsync(p->Ru, 0, nm * sizeof(float), s));
        CTR_CUDA(cudaMemsetAsync(p->v1b, 0, nm * sizeof(float), s));
        CTR_CUDA(cudaMemsetAsync(p->v2b, 0, 2 * nn * sizeof(float), s));
        const bool nonneg = prm.nonneg != 0;                 // Alg. 5
        if (nonneg) CTR_CUDA(cudaMemsetAsync(p->ubar_u, 0, nn * sizeof(float), s));
        if ((st = launch_symbols<float>(p, prm.sigma, prm.tau, c[i], eps, s, nonneg)) != CTR_OK) return st;
        IterArgs<float> &a = args[i];
        a.nonneg = nonneg;
        a.sigma = (float)prm.sigma;
        a.tau = (float)prm.tau;
        a.lam = (float)(alpha[i] / (beta[i] * beta[i]));
        a.inv_beta = (float)(1.0 / beta[i]);
        a.inv_h = (float)(1.0 / p->h);
        p->launches += 2;
        k_axpy<float><<<grid_for(nm, 256, 4096), 256, 0, s>>>((const float *)p->v1b, (const float *)p->Ru, a.sigma, nm,
                                                            (float *)p->y1);
        k_init_y2<float><<<grid_for(nn, 256, 4096), 256, 0, s>>>((const float *)p->u, (const float *)p->v2b, p->n,
                                                               a.sigma * a.tau, a.inv_h, (float *)p->y2);
        CTR_CHECK_LAUNCH("batch init");
        SliceDesc &d = hd[i];
        d.n = p->n;
        d.N = p->N;
        d.M = p->M;
        d.wstride = p->wstride;
        d.orbit = p->orbit ? 1 : 0;
        d.pair_jobs = p->orbit ? p->pair_jobs : 0;
        d.twist = prm.precond == 2 ? 1 : 0;
        d.n_jobs = p->n_jobs;
        d.jobs = p->d_jobs;
        d.ubar = (float4 *)p->ubar;
        d.bp_groups = p->orbit ? p->obp_groups : p->bp_groups;
        d.per_group = p->orbit ? (p->n_jobs + p->obp_groups - 1) / p->obp_groups
                               : (p->N + p->bp_groups - 1) / p->bp_groups;
        bp_tiles(p->n, d.bp_tiles_x, d.bp_tiles_y);
        d.fwd_chunks = fwd_grid_x(p->M);
        d.rpc = fft_rows_per_cta(p->n);
        d.cw = fft_cols_per_cta(p->n, 4);
        d.packed = batch_slice_packed(b, p);
        d.prp = fft_packed_rows_per_cta(p);
        d.pcw = fft_packed_cols_per_cta(p);
        d.geom = p->d_geom;
        d.march = p->d_march;
        d.cbuf = (float2 *)p->cbuf;
        d.tw = (const float2 *)p->d_twiddle;
        d.sym = (const float *)p->sym;
        d.fp.count = (int)p->radices.size();
        for (int r = 0; r < d.fp.count && r < 16; ++r) d.fp.radix[r] = p->radices[r];
        d.u = (float *)p->u;
        d.uT = (float *)p->uT;
        d.y1 = (float *)p->y1;
        d.y2 = (float *)p->y2;
        d.v2b = (float *)p->v2b;
        d.bp_part = (float *)(p->orbit ? p->obp_part : p->bp_part);
        d.bpe = BackprojEpi<float>{};
        d.bpe.out = (float *)p->cbuf;
        d.bpe.complex_out = 1;
        d.bpe.scale = a.inv_beta;
        d.bpe.px = (const float *)p->y2;
        d.bpe.divtau = a.tau;
        d.bpe.outscale = -a.sigma;
        d.bpe.inv_h = a.inv_h;
        d.ub = nonneg ? (float *)p->ubar_u : nullptr;
        if (nonneg) {                                       // u_tmp = bar u - u - sigma (...)
            d.bpe.ub = (const float *)p->ubar_u;
            d.bpe.uu = (const float *)p->u;
        }
        d.fwe = ForwardEpi<float>{};
        d.fwe.mode = 1;
        d.fwe.scale = a.inv_beta;
        d.fwe.sigma = a.sigma;
        d.fwe.Ru = (float *)p->Ru;
        d.fwe.v1b = (float *)p->v1b;
        d.fwe.y1 = (float *)p->y1;
        const float *dd = (const float *)p->desc;
        d.fwe.dw = dd;
        d.fwe.da = dd + nm;
        d.fwe.dlo = dd + 2 * nm;
        d.fwe.dhi = dd + 3 * nm;
        d.sigma = a.sigma;
        d.tau = a.tau;
        d.lam = a.lam;
        d.inv_h = a.inv_h;
        b->launches += p->launches - l0;
    }
    CTR_CUDA(cudaMemcpyAsync(b->d_desc, hd.data(), sizeof(SliceDesc) * ns, cudaMemcpyHostToDevice, s));
    const int body = iters > 0 ? iters - 1 : 0;
    auto one_iteration = [&]() -> ctr_status {
        ctr_status r;
        const int *pre = b->d_prefix;
        const int stride = ns + 1;
        for (int stg : {BS_BP, BS_BP_SYM})
            if ((r = launch_batch_radon(stg, b->d_desc, pre + stg * stride, ns, b->blocks[stg], b->smem[stg], s)) != CTR_OK)
                return r;
        for (int stg = BS_FFT_ROWS; stg <= BS_FFT_ROWS_INV; ++stg)
            if ((r = launch_batch_fft(stg, b->d_desc, pre + stg * stride, ns, b->blocks[stg], b->smem[stg], s)) != CTR_OK) return r;
        for (int stg : {BS_ORBIT, BS_FWD, BS_FWD_SYM})
            if ((r = launch_batch_radon(stg, b->d_desc, pre + stg * stride, ns, b->blocks[stg], 0, s)) != CTR_OK) return r;
        if ((r = launch_batch_tv(b->d_desc, pre + BS_TV * stride, ns, b->blocks[BS_TV], s)) != CTR_OK) return r;
        int nl = 0;
        for (int stg = 0; stg < BS_COUNT; ++stg) nl += b->blocks[stg] > 0 ? 1 : 0;
        b->launches += nl;
        return CTR_OK;
    };
    if (b->mode == 1 && body > 0) {
        // one cooperative launch per iteration; the grid barriers' state starts at zero
        CTR_CUDA(cudaMemsetAsync(b->d_gb, 0, sizeof(GridBarrier), s));
        for (int k = 0; k < body; ++k) {
            if ((st = launch_batch_iteration(b->d_desc, b->d_prefix, ns, b->d_gb, b->spin_limit, b->persist_grid,
                                             b->persist_smem, s)) != CTR_OK)
                return st;
            b->launches++;
        }
        GridBarrier g{};
        CTR_CUDA(cudaMemcpyAsync(&g, b->d_gb, sizeof(g), cudaMemcpyDeviceToHost, s));
        CTR_CUDA(cudaStreamSynchronize(s));
        if (g.status != 0)
            return fail(CTR_ETIMEOUT, "persistent batched iteration: a grid barrier's bounded wait ran out");
    } else {
        const int blk = prm.graph_block;
        std::vector<double> key = {6.0, (double)blk, (double)ns, (double)b->fft_packed};
        for (int stg = 0; stg < BS_COUNT; ++stg) {
            key.push_back((double)b->blocks[stg]);
            key.push_back((double)b->smem[stg]);
        }
        if ((st = run_graphed_in(b->graphs, b->launches, body, blk, one_iteration, s, &key)) != CTR_OK) return st;
    }
    for (int i = 0; i < ns; ++i) {
        ctr_plan *p = b->plans[i];
        const unsigned long long l0 = p->launches;
        if (iters > 0 && (st = pdrq_iteration<float>(p, args[i], true, s)) != CTR_OK) return st;
        if (diags) {
            if (iters <= 0) {
                CTR_CUDA(cudaMemsetAsync(p->du, 0, sizeof(float) * p->n * p->n, s));
                CTR_CUDA(cudaMemsetAsync(p->t1, 0, sizeof(float) * p->N * p->M, s));
                CTR_CUDA(cudaMemsetAsync(p->t2, 0, sizeof(float) * 2 * p->n * p->n, s));
            }
            if ((st = compute_diag<float>(p, alpha[i], beta[i], prm.tau, c[i], iters, &diags[i], s)) != CTR_OK)
                return st;
            if (prm.nonneg) diags[i].gap = diags[i].dual_residual = nan("");   // Alg. 4's saddle problem only
        }
        if (u_out && u_out[i])
            CTR_CUDA(cudaMemcpyAsync(u_out[i], p->u, sizeof(float) * p->n * p->n, cudaMemcpyDeviceToDevice, s));
        b->launches += p->launches - l0;
    }
    return CTR_OK;
}

// A slice's preconditioner stages take the real-input form when the batch's tables use it
// and the first pass reads the backprojection's partial images (the symmetric path, or
// several angle groups): a real input, never the complex buffer the form overwrites.
bool batch_slice_packed(const ctr_batch *b, const ctr_plan *p)
{
    return b->fft_packed && (p->orbit || p->bp_groups > 1);
}

// Block tables and shared-memory sizes of the batched stages.
ctr_status batch_prepare(ctr_batch *b)
{
    const int ns = (int)b->plans.size();
    std::vector<int> pre((size_t)BS_COUNT * (ns + 1), 0);
    for (int stg = 0; stg < BS_COUNT; ++stg) b->smem[stg] = 0;
    for (int i = 0; i < ns; ++i) {
        const ctr_plan *p = b->plans[i];
        int tx, ty;
        bp_tiles(p->n, tx, ty);
        const size_t nn = (size_t)p->n * p->n;
        const bool packed = batch_slice_packed(b, p);
        const int rpc = packed ? fft_packed_rows_per_cta(p) : fft_rows_per_cta(p->n);
        const int cw = fft_cols_per_cta(p->n, 4), pcw = fft_packed_cols_per_cta(p);
        int cnt[BS_COUNT];
        const int t32 = (p->n + 31) / 32;
        cnt[BS_BP] = p->orbit ? 0 : tx * ty * p->bp_groups;
        cnt[BS_BP_SYM] = p->orbit ? tx * ty * p->obp_groups : 0;
        cnt[BS_FFT_ROWS] = (p->n + rpc - 1) / rpc;
        cnt[BS_FFT_COLS] = packed ? (p->n / 2 + 1 + pcw - 1) / pcw : (p->n + cw - 1) / cw;
        cnt[BS_FFT_ROWS_INV] = cnt[BS_FFT_ROWS];
        cnt[BS_ORBIT] = p->orbit ? t32 * t32 : 0;
        cnt[BS_FWD] = p->orbit ? 0 : fwd_grid_x(p->M) * fwd_grid_y(p->N);
        cnt[BS_FWD_SYM] = p->orbit ? fwd_grid_x(p->M) * orbit_fwd_grid_y(p->n_jobs) : 0;
        cnt[BS_TV] = grid_for(nn, 256, 1024);
        for (int stg = 0; stg < BS_COUNT; ++stg) pre[(size_t)stg * (ns + 1) + i + 1] = pre[(size_t)stg * (ns + 1) + i] + cnt[stg];
        const size_t smb = p->orbit ? 0 : bp_smem_bytes(p->wstride), smo = p->orbit ? obp_smem_bytes(p->wstride, (p->n_jobs + p->obp_groups - 1) / p->obp_groups) : 0;
        if (smo > b->smem[BS_BP_SYM]) b->smem[BS_BP_SYM] = smo;
        const size_t smr = packed ? fft_packed_smem(p, 0) : fft_rows_smem(p->n, sizeof(float));
        const size_t smc = packed ? fft_packed_smem(p, 1) : fft_cols_smem(p->n, sizeof(float));
        if (smb > b->smem[BS_BP]) b->smem[BS_BP] = smb;
        if (smr > b->smem[BS_FFT_ROWS]) b->smem[BS_FFT_ROWS] = smr;
        if (smr > b->smem[BS_FFT_ROWS_INV]) b->smem[BS_FFT_ROWS_INV] = smr;
        if (smc > b->smem[BS_FFT_COLS]) b->smem[BS_FFT_COLS] = smc;
    }
    for (int stg = 0; stg < BS_COUNT; ++stg) b->blocks[stg] = pre[(size_t)stg * (ns + 1) + ns];
    CTR_CUDA(cudaMemcpy(b->d_prefix, pre.data(), sizeof(int) * pre.size(), cudaMemcpyHostToDevice));
    ctr_status st = configure_batch_radon(b->smem[BS_BP], b->smem[BS_BP_SYM]);
    if (st == CTR_OK) st = configure_batch_fft(b->smem[BS_FFT_ROWS], b->smem[BS_FFT_COLS]);
    if (st != CTR_OK) return st;
    // the persistent form: every stage's shared memory in one launch, all CTAs resident
    b->persist_smem = 0;
    for (int stg = 0; stg < BS_COUNT; ++stg) b->persist_smem = std::max(b->persist_smem, b->smem[stg]);
    int sms = 0;
    CTR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    b->persist_grid = persist_blocks_per_sm(b->persist_smem) * sms;
    if (b->persist_grid <= 0 && b->mode == 1) b->mode = 0;
    return CTR_OK;
}

#define CTR_INST(T)                                                                                                 \
    template ctr_status dot2<T>(ctr_plan *, const T *, const T *, size_t, double *, cudaStream_t);                  \
    template ctr_status op_grad<T>(ctr_plan *, const T *, T *, cudaStream_t);                                         \
    template ctr_status op_div<T>(ctr_plan *, const T *, T *, cudaStream_t);                                          \
    template ctr_status op_forward<T>(ctr_plan *, const T *, const T *, T *, double, cudaStream_t);                   \
    template ctr_status op_adjoint<T>(ctr_plan *, const T *, T *, double, cudaStream_t);                              \
    template ctr_status power_beta<T>(ctr_plan *, int, double *, cudaStream_t);                                       \
    template ctr_status power_lambda<T>(ctr_plan *, double, double, int, double *, cudaStream_t);                     \
    template ctr_status pdrq_loop<T>(ctr_plan *, double, int, const ctr_params &, double, double, ctr_diag *,         \
                                     cudaStream_t);                                                                   \
    template ctr_status cp_loop<T>(ctr_plan *, double, int, const ctr_params &, double, double, double, ctr_diag *,   \
                                   cudaStream_t);                                                                     \
    template ctr_status prepare_impulse_symbol<T>(ctr_plan *, cudaStream_t);                                          \
    template ctr_status admm_loop<T>(ctr_plan *, double, int, int, double, const ctr_params &, double, double,        \
                                     ctr_diag *, cudaStream_t);                                                       \
    template ctr_status metal_trace<T>(ctr_plan *, const T *, double, int, double, uint8_t *, uint8_t *, cudaStream_t); \
    template ctr_status build_desc_from_data<T>(ctr_plan *, const T *, const uint8_t *, double, double, double,       \
                                                cudaStream_t);                                                        \
    template ctr_status build_desc_from_arrays<T>(ctr_plan *, const T *, const T *, const T *, const T *, double,     \
                                                  cudaStream_t);
CTR_INST(float)
CTR_INST(double)
#undef CTR_INST

}  // namespace ctr
