// Circulant image operators through the 2-D DFT: the inverse-norm preconditioner
// M^{-1} of Alg. 4 (Sec. 4.3.1, 4.4) and the square-root form used by the power
// iteration for c.  out = F^{-1}(sym .* F(in)) with sym real and 1/n^2 folded in.
//
// Three passes over an n x n complex buffer, each a shared-memory mixed-radix
// (4, 2, 3) Stockham FFT:
//   rows   : forward FFT of every row (real input promoted to complex on load)
//   columns: forward FFT of a block of columns, multiply by sym, inverse FFT
//   rows   : inverse FFT of every row, then the epilogue (write, or add to the
//            iterate and also write its transpose for the ray-driven projector).
#include <cmath>

#include "ctr_internal.cuh"

namespace ctr {

ctr_status fft_radices(int n, std::vector<int> &out)
{
    out.clear();
    if (n < 1) return fail(CTR_EINVAL, "FFT length must be >= 1");
    int m = n;
    while (m % 4 == 0) { out.push_back(4); m /= 4; }
    while (m % 2 == 0) { out.push_back(2); m /= 2; }
    while (m % 3 == 0) { out.push_back(3); m /= 3; }
    if (m != 1) return fail(CTR_EUNSUPPORTED, "image size n must be of the form 2^a 3^b for the Fourier preconditioner");
    return CTR_OK;
}

namespace {

constexpr int FFT_THREADS = 256;
constexpr int MAX_PASSES = 16;


template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };

template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b)
{
    T2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { a.x += b.x; a.y += b.y; return a; }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { a.x -= b.x; a.y -= b.y; return a; }

// One Stockham pass of radix R over `cnt` transforms of length n stored with
// leading dimension ld.  Ns = product of the radices already applied.
// sign = -1 forward, +1 inverse.  tw[t] = exp(-2 pi i t / n).
template <typename T, int R>
__device__ __forceinline__ void stockham_pass(const typename C2<T>::type *src, typename C2<T>::type *dst,
                                              int n, int cnt, int ld, int Ns, int sign,
                                              const typename C2<T>::type *__restrict__ tw)
{
    using T2 = typename C2<T>::type;
    const int nr = n / R;
    const int stride_tw = n / (Ns * R);
    for (int b = threadIdx.x; b < cnt * nr; b += blockDim.x) {
        const int t = b / nr;
        const int j = b - t * nr;
        const T2 *in = src + (size_t)t * ld;
        T2 *out = dst + (size_t)t * ld;
        const int k = j % Ns;
        T2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[j + r * nr];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                T2 w = tw[(r * k * stride_tw) % n];
                if (sign > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        const T s = (T)sign;
        if (R == 2) {
            const T2 a = v[0], c = v[1];
            v[0] = cadd(a, c);
            v[1] = csub(a, c);
        } else if (R == 4) {
            const T2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
            const T2 t2 = cadd(v[1], v[3]);
            const T2 d = csub(v[1], v[3]);
            T2 t3;                                  // d * (s i)
            t3.x = -s * d.y;
            t3.y = s * d.x;
            v[0] = cadd(t0, t2);
            v[2] = csub(t0, t2);
            v[1] = cadd(t1, t3);
            v[3] = csub(t1, t3);
        } else if (R == 3) {
            const T c3 = (T)0.86602540378443864676;   // sin(2 pi / 3)
            const T2 a0 = v[0];
            const T2 tt = cadd(v[1], v[2]);
            const T2 d = csub(v[1], v[2]);
            T2 m;
            m.x = a0.x - (T)0.5 * tt.x;
            m.y = a0.y - (T)0.5 * tt.y;
            T2 e;                                   // d * (i s c3)
            e.x = -s * c3 * d.y;
            e.y = s * c3 * d.x;
            v[0] = cadd(a0, tt);
            v[1] = cadd(m, e);
            v[2] = csub(m, e);
        }
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[base + r * Ns] = v[r];
    }
}

// Runs all passes; returns the buffer holding the result (a or b).
template <typename T>
__device__ typename C2<T>::type *fft_smem(typename C2<T>::type *a, typename C2<T>::type *b, int n, int cnt, int ld,
                                          const FftPasses &fp, int sign, const typename C2<T>::type *__restrict__ tw)
{
    using T2 = typename C2<T>::type;
    T2 *src = a, *dst = b;
    int Ns = 1;
    for (int p = 0; p < fp.count; ++p) {
        const int R = fp.radix[p];
        if (R == 4) stockham_pass<T, 4>(src, dst, n, cnt, ld, Ns, sign, tw);
        else if (R == 2) stockham_pass<T, 2>(src, dst, n, cnt, ld, Ns, sign, tw);
        else stockham_pass<T, 3>(src, dst, n, cnt, ld, Ns, sign, tw);
        __syncthreads();
        T2 *tmp = src; src = dst; dst = tmp;
        Ns *= R;
    }
    return src;
}

// Forward row FFTs.  in_real != null: real input promoted to complex; else the
// complex buffer itself is transformed in place.
template <typename T>
__device__ __forceinline__ void fft_rows_fwd_body(const T *__restrict__ in_real, typename C2<T>::type *cbuf, int n,
                                                  int rows_per_cta, const FftPasses &fp,
                                                  const typename C2<T>::type *__restrict__ tw, int bx)
{
    using T2 = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *a = reinterpret_cast<T2 *>(smem_raw);
    T2 *b = a + (size_t)rows_per_cta * n;
    const int r0 = bx * rows_per_cta;
    const int cnt = min(rows_per_cta, n - r0);
    for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
        const size_t g = (size_t)r0 * n + e;
        if (in_real) {
            T2 v;
            v.x = in_real[g];
            v.y = T(0);
            a[e] = v;
        } else {
            a[e] = cbuf[g];
        }
    }
    __syncthreads();
    T2 *res = fft_smem<T>(a, b, n, cnt, n, fp, -1, tw);
    for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) cbuf[(size_t)r0 * n + e] = res[e];
}

template <typename T>
__global__ void __launch_bounds__(FFT_THREADS)
k_fft_rows_fwd(const T *__restrict__ in_real, typename C2<T>::type *cbuf, int n, int rows_per_cta,
               FftPasses fp, const typename C2<T>::type *__restrict__ tw)
{
    fft_rows_fwd_body<T>(in_real, cbuf, n, rows_per_cta, fp, tw, blockIdx.x);
}

// Column FFT, multiply by the real symbol, inverse column FFT (in place on cbuf).
template <typename T>
__device__ __forceinline__ void fft_cols_body(typename C2<T>::type *cbuf, const T *__restrict__ sym, int n, int cw,
                                              const FftPasses &fp, const typename C2<T>::type *__restrict__ tw,
                                              int bx)
{
    using T2 = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ld = n + 1;
    T2 *a = reinterpret_cast<T2 *>(smem_raw);
    T2 *b = a + (size_t)cw * ld;
    const int c0 = bx * cw;
    const int cnt = min(cw, n - c0);
    for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
        const int row = e / cnt, c = e - row * cnt;
        a[(size_t)c * ld + row] = cbuf[(size_t)row * n + c0 + c];
    }
    __syncthreads();
    T2 *res = fft_smem<T>(a, b, n, cnt, ld, fp, -1, tw);
    for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
        const int row = e / cnt, c = e - row * cnt;
        const T m = sym[(size_t)row * n + c0 + c];
        T2 &v = res[(size_t)c * ld + row];
        v.x *= m;
        v.y *= m;
    }
    __syncthreads();
    T2 *other = (res == a) ? b : a;
    T2 *res2 = fft_smem<T>(res, other, n, cnt, ld, fp, +1, tw);
    for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
        const int row = e / cnt, c = e - row * cnt;
        cbuf[(size_t)row * n + c0 + c] = res2[(size_t)c * ld + row];
    }
}

template <typename T>
__global__ void __launch_bounds__(FFT_THREADS)
k_fft_cols(typename C2<T>::type *cbuf, const T *__restrict__ sym, int n, int cw, FftPasses fp,
           const typename C2<T>::type *__restrict__ tw)
{
    fft_cols_body<T>(cbuf, sym, n, cw, fp, tw, blockIdx.x);
}

// Inverse row FFTs and the epilogue on the real part v:
//   mode 0: out = v;  mode 1: out += v.   dout (optional) = v; outT (optional) =
//   transpose of the final out.
template <typename T>
__device__ __forceinline__ void fft_rows_inv_body(const typename C2<T>::type *__restrict__ cbuf, int n,
                                                  int rows_per_cta, const FftPasses &fp,
                                                  const typename C2<T>::type *__restrict__ tw, T *out, int mode,
                                                  T *outT, T *dout, __nv_bfloat16 *outh, __nv_bfloat16 *outTh,
                                                  int bx)
{
    using T2 = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *a = reinterpret_cast<T2 *>(smem_raw);
    T2 *b = a + (size_t)rows_per_cta * n;
    const int r0 = bx * rows_per_cta;
    const int cnt = min(rows_per_cta, n - r0);
    for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) a[e] = cbuf[(size_t)r0 * n + e];
    __syncthreads();
    T2 *res = fft_smem<T>(a, b, n, cnt, n, fp, +1, tw);
    // row-major outputs
    for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
        const size_t g = (size_t)r0 * n + e;
        const T v = res[e].x;
        if (dout) dout[g] = v;
        T o = v;
        if (mode == 1) o += out[g];
        out[g] = o;
        if (outh) outh[g] = __float2bfloat16_rn((float)o);   // bfloat16 operand copy
        res[e].y = o;     // keep the final value for the transposed write
    }
    if (outT || outTh) {
        __syncthreads();
        // column-major writes: consecutive threads take consecutive rows of one column
        for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
            const int col = e / cnt, r = e - col * cnt;
            const T o = res[(size_t)r * n + col].y;
            if (outT) outT[(size_t)col * n + r0 + r] = o;
            if (outTh) outTh[(size_t)col * n + r0 + r] = __float2bfloat16_rn((float)o);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(FFT_THREADS)
k_fft_rows_inv(const typename C2<T>::type *__restrict__ cbuf, int n, int rows_per_cta, FftPasses fp,
               const typename C2<T>::type *__restrict__ tw, T *out, int mode, T *outT, T *dout,
               __nv_bfloat16 *outh, __nv_bfloat16 *outTh)
{
    fft_rows_inv_body<T>(cbuf, n, rows_per_cta, fp, tw, out, mode, outT, dout, outh, outTh, blockIdx.x);
}

__device__ __forceinline__ int find_slice_fft(const int *__restrict__ prefix, int ns, int b)
{
    int lo = 0, hi = ns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Batched preconditioner passes (step B of every slice in one launch each).
__global__ void __launch_bounds__(FFT_THREADS)
k_fft_rows_fwd_batch(const SliceDesc *__restrict__ sd, const int *__restrict__ prefix, int ns)
{
    const int s = find_slice_fft(prefix, ns, blockIdx.x);
    const SliceDesc &d = sd[s];
    fft_rows_fwd_body<float>(nullptr, d.cbuf, d.n, d.rpc, d.fp, d.tw, blockIdx.x - prefix[s]);
}

__global__ void __launch_bounds__(FFT_THREADS)
k_fft_cols_batch(const SliceDesc *__restrict__ sd, const int *__restrict__ prefix, int ns)
{
    const int s = find_slice_fft(prefix, ns, blockIdx.x);
    const SliceDesc &d = sd[s];
    fft_cols_body<float>(d.cbuf, d.sym, d.n, d.cw, d.fp, d.tw, blockIdx.x - prefix[s]);
}

__global__ void __launch_bounds__(FFT_THREADS)
k_fft_rows_inv_batch(const SliceDesc *__restrict__ sd, const int *__restrict__ prefix, int ns)
{
    const int s = find_slice_fft(prefix, ns, blockIdx.x);
    const SliceDesc &d = sd[s];
    fft_rows_inv_body<float>(d.cbuf, d.n, d.rpc, d.fp, d.tw, d.u, 1, d.uT, nullptr, nullptr, nullptr,
                             blockIdx.x - prefix[s]);
}

// Preconditioner symbols (Alg. 4, Sec. 4.3.1), with 1/n^2 of the inverse DFT:
//   sym  = ||xi||_eps / (sigma^2 c + (sigma tau)^2 L ||xi||_eps) / n^2
//   symh = sqrt(||xi||_eps) / n^2
template <typename T>
__global__ void k_symbols(T *sym, T *symh, int n, double sigma, double tau, double c, double eps)
{
    const size_t total = (size_t)n * n;
    const double pi = 3.14159265358979323846;
    const double inv_n2 = 1.0 / ((double)n * (double)n);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const int ii = (2 * i < n) ? i : i - n;    // wrapped signed index (Nyquist sign irrelevant)
        const int jj = (2 * j < n) ? j : j - n;
        const double xi = 2.0 * pi * ii / n, xj = 2.0 * pi * jj / n;
        const double nrm = sqrt(xi * xi + xj * xj + eps * eps);
        const double si = sin(pi * i / n), sj = sin(pi * j / n);
        const double L = 4.0 * si * si + 4.0 * sj * sj;
        sym[e] = (T)(nrm / (sigma * sigma * c + (sigma * tau) * (sigma * tau) * L * nrm) * inv_n2);
        if (symh) symh[e] = (T)(sqrt(nrm) * inv_n2);
    }
}

FftPasses make_passes(const ctr_plan *p)
{
    FftPasses fp;
    fp.count = (int)p->radices.size();
    for (int i = 0; i < fp.count && i < MAX_PASSES; ++i) fp.radix[i] = p->radices[i];
    return fp;
}

int rows_per_cta(const ctr_plan *p)
{
    int r = 2048 / p->n;
    return r < 1 ? 1 : (r > 8 ? 8 : r);
}

int cols_per_cta(const ctr_plan *p)
{
    const size_t c2 = 2 * p->esize;
    for (int cw = 4; cw > 1; cw /= 2)
        if (2 * (size_t)cw * (p->n + 1) * c2 <= 160 * 1024) return cw;
    return 1;
}

}  // namespace

size_t fft_smem_bytes(const ctr_plan *p, int which)
{
    const size_t c2 = 2 * p->esize;
    if (which == 0) return 2 * (size_t)rows_per_cta(p) * p->n * c2;
    return 2 * (size_t)cols_per_cta(p) * (p->n + 1) * c2;
}

template <typename T>
ctr_status launch_circulant(const ctr_plan *p, const T *in_real, bool in_is_cbuf, const T *sym, T *out, int mode,
                            T *outT, T *dout, cudaStream_t s, __nv_bfloat16 *outh, __nv_bfloat16 *outTh)
{
    using T2 = typename C2<T>::type;
    const int n = p->n;
    const FftPasses fp = make_passes(p);
    const T2 *tw = reinterpret_cast<const T2 *>(p->d_twiddle);
    T2 *cb = reinterpret_cast<T2 *>(p->cbuf);
    const int rpc = rows_per_cta(p);
    const int cw = cols_per_cta(p);
    const size_t smr = fft_smem_bytes(p, 0), smc = fft_smem_bytes(p, 1);
    const int gr = (n + rpc - 1) / rpc, gc = (n + cw - 1) / cw;
    p->launches++;
    k_fft_rows_fwd<T><<<gr, FFT_THREADS, smr, s>>>(in_is_cbuf ? nullptr : in_real, cb, n, rpc, fp, tw);
    CTR_CHECK_LAUNCH("k_fft_rows_fwd");
    p->launches++;
    k_fft_cols<T><<<gc, FFT_THREADS, smc, s>>>(cb, sym, n, cw, fp, tw);
    CTR_CHECK_LAUNCH("k_fft_cols");
    p->launches++;
    k_fft_rows_inv<T><<<gr, FFT_THREADS, smr, s>>>(cb, n, rpc, fp, tw, out, mode, outT, dout, outh, outTh);
    CTR_CHECK_LAUNCH("k_fft_rows_inv");
    return CTR_OK;
}

template <typename T>
ctr_status configure_fft(const ctr_plan *p)
{
    const size_t smr = fft_smem_bytes(p, 0), smc = fft_smem_bytes(p, 1);
    ctr_status st = raise_smem_limit(k_fft_rows_fwd<T>, smr);
    if (st == CTR_OK) st = raise_smem_limit(k_fft_rows_inv<T>, smr);
    if (st == CTR_OK) st = raise_smem_limit(k_fft_cols<T>, smc);
    return st;
}

template <typename T>
ctr_status launch_symbols(const ctr_plan *p, double sigma, double tau, double c, double eps, cudaStream_t s)
{
    const size_t total = (size_t)p->n * p->n;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    p->launches++;
    k_symbols<T><<<blocks, 256, 0, s>>>((T *)p->sym, (T *)p->symh, p->n, sigma, tau, c, eps);
    CTR_CHECK_LAUNCH("k_symbols");
    return CTR_OK;
}

template ctr_status launch_circulant<float>(const ctr_plan *, const float *, bool, const float *, float *, int, float *, float *, cudaStream_t, __nv_bfloat16 *, __nv_bfloat16 *);
template ctr_status launch_circulant<double>(const ctr_plan *, const double *, bool, const double *, double *, int, double *, double *, cudaStream_t, __nv_bfloat16 *, __nv_bfloat16 *);
ctr_status configure_batch_fft(size_t rows_smem, size_t cols_smem)
{
    ctr_status st = raise_smem_limit(k_fft_rows_fwd_batch, rows_smem);
    if (st == CTR_OK) st = raise_smem_limit(k_fft_rows_inv_batch, rows_smem);
    if (st == CTR_OK) st = raise_smem_limit(k_fft_cols_batch, cols_smem);
    return st;
}

// One batched preconditioner pass over all slices.
ctr_status launch_batch_fft(int stage, const SliceDesc *sd, const int *prefix, int ns, int blocks, size_t smem,
                            cudaStream_t s)
{
    if (blocks <= 0) return CTR_OK;
    switch (stage) {
    case BS_FFT_ROWS: k_fft_rows_fwd_batch<<<blocks, FFT_THREADS, smem, s>>>(sd, prefix, ns); break;
    case BS_FFT_COLS: k_fft_cols_batch<<<blocks, FFT_THREADS, smem, s>>>(sd, prefix, ns); break;
    case BS_FFT_ROWS_INV: k_fft_rows_inv_batch<<<blocks, FFT_THREADS, smem, s>>>(sd, prefix, ns); break;
    default: return fail(CTR_EINVAL, "not an FFT stage");
    }
    CTR_CHECK_LAUNCH("batched FFT stage");
    return CTR_OK;
}

int fft_rows_per_cta(int n)
{
    int r = 2048 / n;
    return r < 1 ? 1 : (r > 8 ? 8 : r);
}

int fft_cols_per_cta(int n, size_t esize)
{
    for (int cw = 4; cw > 1; cw /= 2)
        if (2 * (size_t)cw * (n + 1) * 2 * esize <= 160 * 1024) return cw;
    return 1;
}

template ctr_status configure_fft<float>(const ctr_plan *);
template ctr_status configure_fft<double>(const ctr_plan *);
template ctr_status launch_symbols<float>(const ctr_plan *, double, double, double, double, cudaStream_t);
template ctr_status launch_symbols<double>(const ctr_plan *, double, double, double, double, cudaStream_t);

// ------------------------------------------------------------------------------
// precond_apply_static: the FP32 preconditioner without any device allocation.
// Its scratch (the complex FFT buffer, the symbol and the twiddles for one image of
// up to STATIC_MAX_N x STATIC_MAX_N) lives in file-scope __device__ arrays that every
// GPU loading this library holds until the process exits (12 MiB + 8 KiB).  Host
// code cannot use these names as device addresses, so the addresses are looked up
// once per device with cudaGetSymbolAddress, with that device current, on the
// first call made on it.  All calls share the arrays: calls that overlap on the GPU
// (different streams, or different host threads) race on them.
// ------------------------------------------------------------------------------
namespace {

constexpr int STATIC_MAX_N = 1024;
constexpr int STATIC_MAX_DEVICES = 64;

static __device__ __align__(256) float2 g_static_cbuf[STATIC_MAX_N * STATIC_MAX_N];
static __device__ __align__(256) float g_static_sym[STATIC_MAX_N * STATIC_MAX_N];
static __device__ __align__(256) float2 g_static_tw[STATIC_MAX_N];

struct StaticScratch {
    float2 *cbuf = nullptr;
    float *sym = nullptr;
    float2 *tw = nullptr;
    bool ready = false;
};
static StaticScratch g_scratch[STATIC_MAX_DEVICES];

// tw[t] = exp(-2 pi i t/n), computed in double and rounded to float
__global__ void k_static_twiddles(float2 *tw, int n)
{
    const double pi = 3.14159265358979323846;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        tw[t] = make_float2((float)cos(2.0 * pi * t / n), (float)(-sin(2.0 * pi * t / n)));
}

// Set-up for the current device (first call on it): symbol addresses and the
// shared-memory limits of the FFT kernels.  Not thread-safe against a concurrent
// first call on the same device.
ctr_status static_setup(int dev)
{
    StaticScratch &s = g_scratch[dev];
    if (s.ready) return CTR_OK;
    CTR_CUDA(cudaGetSymbolAddress((void **)&s.cbuf, g_static_cbuf));
    CTR_CUDA(cudaGetSymbolAddress((void **)&s.sym, g_static_sym));
    CTR_CUDA(cudaGetSymbolAddress((void **)&s.tw, g_static_tw));
    const int smax = 2 * 4 * (STATIC_MAX_N + 1) * (int)sizeof(float2);   // column kernel at n = 1024
    ctr_status st = raise_smem_limit(k_fft_cols<float>, smax);
    if (st == CTR_OK) st = raise_smem_limit(k_fft_rows_fwd<float>, smax);
    if (st == CTR_OK) st = raise_smem_limit(k_fft_rows_inv<float>, smax);
    if (st != CTR_OK) return st;
    s.ready = true;
    return CTR_OK;
}

}  // namespace

}  // namespace ctr

extern "C" ctr_status precond_apply_static(int n, double sigma, double tau, double c, double eps, const float *y_dev,
                                           float *x_dev, void *stream)
{
    using namespace ctr;
    if (n < 1 || n > STATIC_MAX_N)
        return fail(CTR_EINVAL, "precond_apply_static: n must be in [1, " + std::to_string(STATIC_MAX_N) +
                                    "] (the size of its static scratch)");
    if (!y_dev || !x_dev) return fail(CTR_EINVAL, "precond_apply_static: null buffer");
    if (!(sigma > 0) || !(tau > 0) || !(c > 0) || !(eps > 0) || !std::isfinite(sigma) || !std::isfinite(tau) ||
        !std::isfinite(c) || !std::isfinite(eps))
        return fail(CTR_EINVAL, "precond_apply_static: sigma, tau, c and eps must be finite and > 0");
    FftPasses fp;
    {
        int m = n, cnt = 0;
        while (m % 4 == 0) { fp.radix[cnt++] = 4; m /= 4; }
        while (m % 2 == 0) { fp.radix[cnt++] = 2; m /= 2; }
        while (m % 3 == 0) { fp.radix[cnt++] = 3; m /= 3; }
        if (m != 1) return fail(CTR_EUNSUPPORTED, "precond_apply_static: n must be of the form 2^a 3^b");
        fp.count = cnt;
    }
    int dev = -1;
    CTR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= STATIC_MAX_DEVICES) return fail(CTR_EUNSUPPORTED, "precond_apply_static: device index too large");
    ctr_status st = static_setup(dev);
    if (st != CTR_OK) return st;
    const StaticScratch &s = g_scratch[dev];
    cudaStream_t str = (cudaStream_t)stream;
    // the same three FFT passes as precond_apply, with every scratch in the static arrays
    k_static_twiddles<<<(n + 255) / 256, 256, 0, str>>>(s.tw, n);
    const size_t nn = (size_t)n * n;
    int blocks = (int)((nn + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_symbols<float><<<blocks, 256, 0, str>>>(s.sym, nullptr, n, sigma, tau, c, eps);
    int rpc = 2048 / n;
    rpc = rpc < 1 ? 1 : (rpc > 8 ? 8 : rpc);
    int cw = 1;
    for (int w = 4; w > 1; w /= 2)
        if (2 * (size_t)w * (n + 1) * sizeof(float2) <= 160 * 1024) { cw = w; break; }
    const size_t smr = 2 * (size_t)rpc * n * sizeof(float2), smc = 2 * (size_t)cw * (n + 1) * sizeof(float2);
    const int gr = (n + rpc - 1) / rpc, gc = (n + cw - 1) / cw;
    k_fft_rows_fwd<float><<<gr, FFT_THREADS, smr, str>>>(y_dev, s.cbuf, n, rpc, fp, s.tw);
    k_fft_cols<float><<<gc, FFT_THREADS, smc, str>>>(s.cbuf, s.sym, n, cw, fp, s.tw);
    k_fft_rows_inv<float><<<gr, FFT_THREADS, smr, str>>>(s.cbuf, n, rpc, fp, s.tw, x_dev, 0, nullptr, nullptr,
                                                         nullptr, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "precond_apply_static launch");
    return CTR_OK;
}
