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
#include <cstring>

#include "ctr_internal.cuh"

namespace ctr {

ctr_status fft_radices(int n, std::vector<int> &out)
{
    out.clear();
    if (n < 1) return fail(CTR_EINVAL, "FFT length must be >= 1");
    int m = n;
    while (m % 8 == 0) { out.push_back(8); m /= 8; }
    while (m % 4 == 0) { out.push_back(4); m /= 4; }
    while (m % 2 == 0) { out.push_back(2); m /= 2; }
    while (m % 3 == 0) { out.push_back(3); m /= 3; }
    if (m != 1) return fail(CTR_EUNSUPPORTED, "image size n must be of the form 2^a 3^b for the Fourier preconditioner");
    return CTR_OK;
}

int ramp_length(int M)
{
    const int need = 2 * (M > 1 ? M : 1) - 1;
    int best = 0;
    for (long long p2 = 1; p2 < 4LL * need; p2 *= 2)
        for (long long v = p2; v < 4LL * need; v *= 3)
            if (v >= need && (best == 0 || v < best)) best = (int)v;
    return best;
}

namespace {

#ifndef CTR_FFT_THREADS
#define CTR_FFT_THREADS 256
#endif
#ifndef CTR_FFT_POINTS
#define CTR_FFT_POINTS 1024
#endif
constexpr int FFT_THREADS = CTR_FFT_THREADS;
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

// exp(-2 pi i r / N) for the twisted column pass, 0 <= r < N = n^2 (r and N are exact
// in FP32 up to n = 4096; beyond, their rounding moves the phase by at most about
// 2 pi 2^-24, the FP32 rounding of the factor itself)
__device__ __forceinline__ float2 twist_factor(float, int r, int N)
{
    float sn, cs;
    sincospif(2.0f * (float)r / (float)N, &sn, &cs);
    return make_float2(cs, -sn);
}
__device__ __forceinline__ double2 twist_factor(double, int r, int N)
{
    double sn, cs;
    sincospi(2.0 * (double)r / (double)N, &sn, &cs);
    return make_double2(cs, -sn);
}
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { a.x -= b.x; a.y -= b.y; return a; }

// x / d for 0 <= x, x d < 2^32 through a multiply-high: m = floor(2^32 / d) + 1
// (d = 1 handled apart).  Exact under that bound (x, d <= 2^14 here).
__device__ __forceinline__ unsigned div_magic(unsigned d) { return d <= 1 ? 0u : 0xFFFFFFFFu / d + 1u; }
__device__ __forceinline__ int fast_div(int x, int d, unsigned m) { return d <= 1 ? x : (int)__umulhi((unsigned)x, m); }

// 4-point DFT with sign s (y_m = sum_k x_k e^{s 2 pi i k m / 4}), in place.
template <typename T, typename T2>
__device__ __forceinline__ void dft4(T2 &x0, T2 &x1, T2 &x2, T2 &x3, T s)
{
    const T2 t0 = cadd(x0, x2), t1 = csub(x0, x2);
    const T2 t2 = cadd(x1, x3);
    const T2 d = csub(x1, x3);
    T2 t3;                                           // d * (s i)
    t3.x = -s * d.y;
    t3.y = s * d.x;
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}

// One Stockham pass of radix R over `cnt` transforms of length n stored with
// leading dimension ld.  Ns = product of the radices already applied.
// sign = -1 forward, +1 inverse.  tw[t] = exp(-2 pi i t / n), staged in shared memory.
template <typename T, int R>
__device__ __forceinline__ void stockham_pass(const typename C2<T>::type *src, typename C2<T>::type *dst,
                                              int n, int cnt, int ld, int Ns, int sign,
                                              const typename C2<T>::type *__restrict__ tw)
{
    using T2 = typename C2<T>::type;
    const int nr = n / R;
    const int stride_tw = n / (Ns * R);
    const unsigned m_nr = div_magic(nr), m_ns = div_magic(Ns);
    const T s = (T)sign;
    for (int b = threadIdx.x; b < cnt * nr; b += blockDim.x) {
        const int t = cnt == 1 ? 0 : fast_div(b, nr, m_nr);
        const int j = b - t * nr;
        const int jq = fast_div(j, Ns, m_ns);
        const int k = j - jq * Ns;
        const T2 *in = src + (size_t)t * ld;
        T2 *out = dst + (size_t)t * ld;
        T2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[j + r * nr];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                T2 w = tw[r * k * stride_tw];           // r k stride_tw < R Ns n/(Ns R) = n
                if (sign > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        if (R == 2) {
            const T2 a = v[0], c = v[1];
            v[0] = cadd(a, c);
            v[1] = csub(a, c);
        } else if (R == 4) {
            dft4<T, T2>(v[0], v[1], v[2], v[3], s);
        } else if (R == 8) {
            // X_{2m} = DFT4(v_k + v_{k+4})_m, X_{2m+1} = DFT4((v_k - v_{k+4}) W^k)_m, W = e^{s i pi/4}
            const T h = (T)0.70710678118654752440;
            T2 a[4], c[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = cadd(v[q], v[q + 4]);
                c[q] = csub(v[q], v[q + 4]);
            }
            T2 e;
            e.x = h * (c[1].x - s * c[1].y);             // c1 (1 + s i) h
            e.y = h * (c[1].y + s * c[1].x);
            c[1] = e;
            e.x = -s * c[2].y;                           // c2 (s i)
            e.y = s * c[2].x;
            c[2] = e;
            e.x = -h * (c[3].x + s * c[3].y);            // c3 (-1 + s i) h
            e.y = h * (s * c[3].x - c[3].y);
            c[3] = e;
            dft4<T, T2>(a[0], a[1], a[2], a[3], s);
            dft4<T, T2>(c[0], c[1], c[2], c[3], s);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                v[2 * q] = a[q];
                v[2 * q + 1] = c[q];
            }
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
        const int base = jq * Ns * R + k;
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
        if (R == 8) stockham_pass<T, 8>(src, dst, n, cnt, ld, Ns, sign, tw);
        else if (R == 4) stockham_pass<T, 4>(src, dst, n, cnt, ld, Ns, sign, tw);
        else if (R == 2) stockham_pass<T, 2>(src, dst, n, cnt, ld, Ns, sign, tw);
        else stockham_pass<T, 3>(src, dst, n, cnt, ld, Ns, sign, tw);
        __syncthreads();
        T2 *tmp = src; src = dst; dst = tmp;
        Ns *= R;
    }
    return src;
}

// Element-wise copy phase of a CTA: store(e, load(e)) for e in [0, total), with
// LD_UNROLL independent loads in flight per thread (the data are L2-resident and
// the kernels few-warp: latency, not bandwidth, bounds these phases).
constexpr int LD_UNROLL = 4;
template <typename L, typename W>
__device__ __forceinline__ void staged_copy(int total, L load, W store)
{
    for (int e0 = threadIdx.x; e0 < total; e0 += LD_UNROLL * blockDim.x) {
        decltype(load(0)) v[LD_UNROLL];
#pragma unroll
        for (int q = 0; q < LD_UNROLL; ++q) {
            const int e = e0 + q * blockDim.x;
            if (e < total) v[q] = load(e);
        }
#pragma unroll
        for (int q = 0; q < LD_UNROLL; ++q) {
            const int e = e0 + q * blockDim.x;
            if (e < total) store(e, v[q]);
        }
    }
}

// The twiddle table copied into shared memory (read by every pass of the CTA).
template <typename T2>
__device__ __forceinline__ void stage_twiddles(T2 *stw, const T2 *__restrict__ tw, int n)
{
    for (int t = threadIdx.x; t < n; t += blockDim.x) stw[t] = tw[t];
}

// Input of the forward row pass.  part != null: the angle-group partial images of
// the backprojection, summed in group order and passed through the backprojection
// epilogue (this fuses the group reduction into the pass); else in_real != null: a
// real image; else the complex buffer itself.
template <typename T>
struct RowsInput {
    const T *in_real;
    const T *part;
    int groups;
    int orbit;                // part holds the symmetric path's partial planes (FP32)
    BackprojEpi<T> epi;
};

// The real input of the forward row pass at (row, col) for the part / in_real sources.
template <typename T>
__device__ __forceinline__ T rows_input_value(const RowsInput<T> &src, int n, int row, int col)
{
    const size_t e = (size_t)row * n + col;
    if (!src.part) return src.in_real[e];
    T acc;
    if constexpr (sizeof(T) == 4) {
        if (src.orbit) acc = orbit_fold(src.part, src.groups, n, row, col);
    }
    if (!(sizeof(T) == 4 && src.orbit)) {
        const size_t nn = (size_t)n * n;
        const T *pp = src.part + e;
        acc = pp[0];
#pragma unroll
        for (int z = 1; z < MAX_BP_GROUPS; ++z)
            if (z < src.groups) acc += pp[(size_t)z * nn];
    }
    return bp_epilogue_value(src.epi, n, row, col, acc);
}

// Real-input form of the forward row pass (for real images and real even symbols):
// rows 2c and 2c + 1 of the CTA's rows go through one complex FFT as z = x_a + i x_b,
// and X_a(k) = (Z(k) + conj Z(n-k)) / 2, X_b(k) = (Z(k) - conj Z(n-k)) / (2i) are kept for
// k = 0 .. n/2 only (the rest is their conjugate mirror): cbuf holds n rows of
// H = n/2 + 1 coefficients.  Inputs: the part or in_real sources (never cbuf itself,
// whose rows the packed output would overwrite).
template <typename T>
__device__ __forceinline__ void fft_rows_fwd_packed_body(const RowsInput<T> &src, typename C2<T>::type *cbuf, int n,
                                                         int rows_per_cta, const FftPasses &fp,
                                                         const typename C2<T>::type *__restrict__ tw, int bx)
{
    using T2 = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int cmax = rows_per_cta / 2;
    T2 *a = reinterpret_cast<T2 *>(smem_raw);
    T2 *b = a + (size_t)cmax * n;
    T2 *stw = b + (size_t)cmax * n;
    stage_twiddles(stw, tw, n);
    const int r0 = bx * rows_per_cta;
    const int cnt = min(rows_per_cta, n - r0);
    const int cc = (cnt + 1) / 2;
    const int H = n / 2 + 1;
    const unsigned mn = div_magic(n);
    bool folded = false;
    if constexpr (sizeof(T) == 4) {
        if (src.part && src.orbit && (n & 3) == 0) {
            // the fold of the partial planes four columns at a time (16-byte loads), then
            // the step-A epilogue per pixel
            const int q = n / 4;
            const unsigned mq = div_magic(q);
            for (int e4 = threadIdx.x; e4 < cc * q; e4 += blockDim.x) {
                const int c = fast_div(e4, q, mq), j = 4 * (e4 - c * q);
                const int ra = r0 + 2 * c;
                const bool two = ra + 1 < r0 + cnt;
                const float4 fa = orbit_fold4(src.part, src.groups, n, ra, j);
                const float4 fb = two ? orbit_fold4(src.part, src.groups, n, ra + 1, j) : make_float4(0.f, 0.f, 0.f, 0.f);
                T2 *dst = a + (size_t)c * n + j;
                dst[0].x = bp_epilogue_value(src.epi, n, ra, j, fa.x);
                dst[1].x = bp_epilogue_value(src.epi, n, ra, j + 1, fa.y);
                dst[2].x = bp_epilogue_value(src.epi, n, ra, j + 2, fa.z);
                dst[3].x = bp_epilogue_value(src.epi, n, ra, j + 3, fa.w);
                dst[0].y = two ? bp_epilogue_value(src.epi, n, ra + 1, j, fb.x) : T(0);
                dst[1].y = two ? bp_epilogue_value(src.epi, n, ra + 1, j + 1, fb.y) : T(0);
                dst[2].y = two ? bp_epilogue_value(src.epi, n, ra + 1, j + 2, fb.z) : T(0);
                dst[3].y = two ? bp_epilogue_value(src.epi, n, ra + 1, j + 3, fb.w) : T(0);
            }
            folded = true;
        }
    }
    if (!folded)
        staged_copy(cc * n, [&](int e) {
            const int c = fast_div(e, n, mn), j = e - c * n;
            const int ra = r0 + 2 * c;
            T2 v;
            v.x = rows_input_value(src, n, ra, j);
            v.y = ra + 1 < r0 + cnt ? rows_input_value(src, n, ra + 1, j) : T(0);
            return v;
        }, [&](int e, T2 v) { a[e] = v; });
    __syncthreads();
    T2 *res = fft_smem<T>(a, b, n, cc, n, fp, -1, stw);
    const unsigned mh = div_magic(H);
    for (int e = threadIdx.x; e < cc * H; e += blockDim.x) {
        const int c = fast_div(e, H, mh), k = e - c * H;
        const T2 z = res[(size_t)c * n + k], zm = res[(size_t)c * n + (k == 0 ? 0 : n - k)];
        const int ra = r0 + 2 * c;
        T2 xa, xb;
        xa.x = T(0.5) * (z.x + zm.x);
        xa.y = T(0.5) * (z.y - zm.y);
        xb.x = T(0.5) * (z.y + zm.y);
        xb.y = T(0.5) * (zm.x - z.x);
        cbuf[(size_t)ra * H + k] = xa;
        if (ra + 1 < r0 + cnt) cbuf[(size_t)(ra + 1) * H + k] = xb;
    }
}

template <typename T>
__global__ void __launch_bounds__(FFT_THREADS)
k_fft_rows_fwd_packed(RowsInput<T> src, typename C2<T>::type *cbuf, int n, int rows_per_cta, FftPasses fp,
                      const typename C2<T>::type *__restrict__ tw)
{
    fft_rows_fwd_packed_body<T>(src, cbuf, n, rows_per_cta, fp, tw, blockIdx.x);
}

// Forward row FFTs (in place on cbuf).
template <typename T>
__device__ __forceinline__ void fft_rows_fwd_body(const RowsInput<T> &src, typename C2<T>::type *cbuf, int n,
                                                  int rows_per_cta, const FftPasses &fp,
                                                  const typename C2<T>::type *__restrict__ tw, int bx)
{
    using T2 = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *a = reinterpret_cast<T2 *>(smem_raw);
    T2 *b = a + (size_t)rows_per_cta * n;
    T2 *stw = b + (size_t)rows_per_cta * n;
    stage_twiddles(stw, tw, n);
    const int r0 = bx * rows_per_cta;
    const int cnt = min(rows_per_cta, n - r0);
    const size_t g0 = (size_t)r0 * n;
    const auto put = [&](int e, T2 v) { a[e] = v; };
    if (src.part) {
        const size_t nn = (size_t)n * n;
        const unsigned mn = div_magic(n);
        staged_copy(cnt * n, [&](int e) {
            const int di = fast_div(e, n, mn);
            T acc;
            if constexpr (sizeof(T) == 4) {
                if (src.orbit) acc = orbit_fold(src.part, src.groups, n, r0 + di, e - di * n);
            }
            if (!(sizeof(T) == 4 && src.orbit)) {
                const T *pp = src.part + g0 + e;
                acc = pp[0];
#pragma unroll
                for (int z = 1; z < MAX_BP_GROUPS; ++z)
                    if (z < src.groups) acc += pp[(size_t)z * nn];
            }
            T2 v;
            v.x = bp_epilogue_value(src.epi, n, r0 + di, e - di * n, acc);
            v.y = T(0);
            return v;
        }, put);
    } else if (src.in_real) {
        staged_copy(cnt * n, [&](int e) {
            T2 v;
            v.x = src.in_real[g0 + e];
            v.y = T(0);
            return v;
        }, put);
    } else {
        staged_copy(cnt * n, [&](int e) { return cbuf[g0 + e]; }, put);
    }
    __syncthreads();
    T2 *res = fft_smem<T>(a, b, n, cnt, n, fp, -1, stw);
    staged_copy(cnt * n, [&](int e) { return res[e]; }, [&](int e, T2 v) { cbuf[g0 + e] = v; });
}

template <typename T>
__global__ void __launch_bounds__(FFT_THREADS)
k_fft_rows_fwd(RowsInput<T> src, typename C2<T>::type *cbuf, int n, int rows_per_cta, FftPasses fp,
               const typename C2<T>::type *__restrict__ tw)
{
    fft_rows_fwd_body<T>(src, cbuf, n, rows_per_cta, fp, tw, blockIdx.x);
}

// Column FFT, multiply by the real symbol, inverse column FFT (in place on cbuf);
// sym == null: the forward column FFT only.
// twist: the 1-D DFT of length N = n^2 of the image flattened as t = i + n j (the
// circulant preconditioner) instead of the 2-D DFT.  With k = kB + n kA,
//   sum_t x_t e^{-2 pi i t k / N} = sum_i e^{-2 pi i i kA / n} [ e^{-2 pi i i kB / N} sum_j x_ij e^{-2 pi i j kB / n} ],
// so the row pass is unchanged, the column pass multiplies element (i, kB) by
// e^{-2 pi i i kB / N} before its forward transform (and by the conjugate after the
// inverse one), and F_1(x)_k lands at (kA, kB), i.e. at flat position k.
// ncols / ldg: the columns present and the row stride of cbuf (n and n, or H = n/2 + 1
// for both in the real-input form; the symbol keeps its n x n layout).
template <typename T>
__device__ __forceinline__ void fft_cols_body(typename C2<T>::type *cbuf, const T *__restrict__ sym, int n, int cw,
                                              const FftPasses &fp, const typename C2<T>::type *__restrict__ tw,
                                              int bx, int twist = 0, int ncols = 0, int ldg = 0)
{
    using T2 = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ld = n + 1;
    if (ncols <= 0) ncols = n;
    if (ldg <= 0) ldg = n;
    T2 *a = reinterpret_cast<T2 *>(smem_raw);
    T2 *b = a + (size_t)cw * ld;
    T2 *stw = b + (size_t)cw * ld;
    stage_twiddles(stw, tw, n);
    const int c0 = bx * cw;
    const int cnt = min(cw, ncols - c0);
    const unsigned mc = div_magic(cnt);
    // element e: row e / cnt, column c0 + e % cnt (consecutive threads: consecutive columns)
    staged_copy(cnt * n, [&](int e) {
        const int row = fast_div(e, cnt, mc);
        return cbuf[(size_t)row * ldg + c0 + (e - row * cnt)];
    }, [&](int e, T2 v) {
        const int row = fast_div(e, cnt, mc);
        if (twist) v = cmul(v, twist_factor(T(0), row * (c0 + e - row * cnt), n * n));
        a[(size_t)(e - row * cnt) * ld + row] = v;
    });
    __syncthreads();
    T2 *res = fft_smem<T>(a, b, n, cnt, ld, fp, -1, stw);
    if (!sym) {                                   // forward transform only: write F back
        staged_copy(cnt * n, [&](int e) {
            const int row = fast_div(e, cnt, mc);
            return res[(size_t)(e - row * cnt) * ld + row];
        }, [&](int e, T2 v) {
            const int row = fast_div(e, cnt, mc);
            cbuf[(size_t)row * ldg + c0 + (e - row * cnt)] = v;
        });
        return;
    }
    staged_copy(cnt * n, [&](int e) {
        const int row = fast_div(e, cnt, mc);
        return sym[(size_t)row * n + c0 + (e - row * cnt)];
    }, [&](int e, T m) {
        const int row = fast_div(e, cnt, mc);
        T2 &v = res[(size_t)(e - row * cnt) * ld + row];
        v.x *= m;
        v.y *= m;
    });
    __syncthreads();
    T2 *other = (res == a) ? b : a;
    T2 *res2 = fft_smem<T>(res, other, n, cnt, ld, fp, +1, stw);
    staged_copy(cnt * n, [&](int e) {
        const int row = fast_div(e, cnt, mc);
        return res2[(size_t)(e - row * cnt) * ld + row];
    }, [&](int e, T2 v) {
        const int row = fast_div(e, cnt, mc);
        if (twist) {
            T2 w = twist_factor(T(0), row * (c0 + e - row * cnt), n * n);
            w.y = -w.y;
            v = cmul(v, w);
        }
        cbuf[(size_t)row * ldg + c0 + (e - row * cnt)] = v;
    });
}

template <typename T>
__global__ void __launch_bounds__(FFT_THREADS)
k_fft_cols(typename C2<T>::type *cbuf, const T *__restrict__ sym, int n, int cw, FftPasses fp,
           const typename C2<T>::type *__restrict__ tw, int twist)
{
    fft_cols_body<T>(cbuf, sym, n, cw, fp, tw, blockIdx.x, twist);
}

// The column pass of the real-input form: the H = n/2 + 1 stored columns.
template <typename T>
__global__ void __launch_bounds__(FFT_THREADS)
k_fft_cols_packed(typename C2<T>::type *cbuf, const T *__restrict__ sym, int n, int cw, FftPasses fp,
                  const typename C2<T>::type *__restrict__ tw)
{
    fft_cols_body<T>(cbuf, sym, n, cw, fp, tw, blockIdx.x, 0, n / 2 + 1, n / 2 + 1);
}

// Inverse of the real-input form: rows 2c and 2c + 1 rebuilt from their H stored
// coefficients (X(k) = conj X(n-k) beyond n/2), transformed together as
// Z = X_a + i X_b, real part -> row 2c, imaginary part -> row 2c + 1; then the same
// epilogue as fft_rows_inv_body (the final values staged in the spare buffer for the
// transposed writes).
template <typename T>
__device__ __forceinline__ void fft_rows_inv_packed_body(const typename C2<T>::type *__restrict__ cbuf, int n,
                                                         int rows_per_cta, const FftPasses &fp,
                                                         const typename C2<T>::type *__restrict__ tw, T *out,
                                                         int mode, T *outT, T *dout, __nv_bfloat16 *outh,
                                                         __nv_bfloat16 *outTh, int bx)
{
    using T2 = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int cmax = rows_per_cta / 2;
    T2 *a = reinterpret_cast<T2 *>(smem_raw);
    T2 *b = a + (size_t)cmax * n;
    T2 *stw = b + (size_t)cmax * n;
    stage_twiddles(stw, tw, n);
    const int r0 = bx * rows_per_cta;
    const int cnt = min(rows_per_cta, n - r0);
    const int cc = (cnt + 1) / 2;
    const int H = n / 2 + 1, half = n / 2;
    const unsigned mn = div_magic(n);
    staged_copy(cc * n, [&](int e) {
        const int c = fast_div(e, n, mn), k = e - c * n;
        const int ra = r0 + 2 * c;
        const bool lo = k <= half;
        const int kk = lo ? k : n - k;
        T2 xa = cbuf[(size_t)ra * H + kk];
        T2 xb;
        xb.x = T(0);
        xb.y = T(0);
        if (ra + 1 < r0 + cnt) xb = cbuf[(size_t)(ra + 1) * H + kk];
        if (!lo) {
            xa.y = -xa.y;
            xb.y = -xb.y;
        }
        T2 z;
        z.x = xa.x - xb.y;
        z.y = xa.y + xb.x;
        return z;
    }, [&](int e, T2 v) { a[e] = v; });
    __syncthreads();
    T2 *res = fft_smem<T>(a, b, n, cc, n, fp, +1, stw);
    T *fin = reinterpret_cast<T *>(res == a ? b : a);              // final values, [local row][col]
    const size_t g0 = (size_t)r0 * n;
    staged_copy(cnt * n, [&](int e) { return mode == 1 ? out[g0 + e] : T(0); }, [&](int e, T prev) {
        const int rl = fast_div(e, n, mn), j = e - rl * n;
        const T2 z = res[(size_t)(rl >> 1) * n + j];
        const T v = (rl & 1) ? z.y : z.x;
        if (dout) dout[g0 + e] = v;
        const T o = v + prev;
        out[g0 + e] = o;
        if (outh) outh[g0 + e] = __float2bfloat16_rn((float)o);
        fin[e] = o;
    });
    if (outT || outTh) {
        __syncthreads();
        const unsigned mc = div_magic(cnt);
        for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
            const int col = fast_div(e, cnt, mc), r = e - col * cnt;
            const T o = fin[(size_t)r * n + col];
            if (outT) outT[(size_t)col * n + r0 + r] = o;
            if (outTh) outTh[(size_t)col * n + r0 + r] = __float2bfloat16_rn((float)o);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(FFT_THREADS)
k_fft_rows_inv_packed(const typename C2<T>::type *__restrict__ cbuf, int n, int rows_per_cta, FftPasses fp,
                      const typename C2<T>::type *__restrict__ tw, T *out, int mode, T *outT, T *dout,
                      __nv_bfloat16 *outh, __nv_bfloat16 *outTh)
{
    fft_rows_inv_packed_body<T>(cbuf, n, rows_per_cta, fp, tw, out, mode, outT, dout, outh, outTh, blockIdx.x);
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
    T2 *stw = b + (size_t)rows_per_cta * n;
    stage_twiddles(stw, tw, n);
    const int r0 = bx * rows_per_cta;
    const int cnt = min(rows_per_cta, n - r0);
    const size_t g0 = (size_t)r0 * n;
    staged_copy(cnt * n, [&](int e) { return cbuf[g0 + e]; }, [&](int e, T2 v) { a[e] = v; });
    __syncthreads();
    T2 *res = fft_smem<T>(a, b, n, cnt, n, fp, +1, stw);
    // row-major outputs
    staged_copy(cnt * n, [&](int e) { return mode == 1 ? out[g0 + e] : T(0); }, [&](int e, T prev) {
        const T v = res[e].x;
        if (dout) dout[g0 + e] = v;
        const T o = v + prev;
        out[g0 + e] = o;
        if (outh) outh[g0 + e] = __float2bfloat16_rn((float)o);   // bfloat16 operand copy
        res[e].y = o;     // keep the final value for the transposed write
    });
    if (outT || outTh) {
        __syncthreads();
        // column-major writes: consecutive threads take consecutive rows of one column
        const unsigned mc = div_magic(cnt);
        for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
            const int col = fast_div(e, cnt, mc), r = e - col * cnt;
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

// ---------------------------------------------------------------------------------------
// Warp-level transforms for n = 32 V (V = 8, 16, 32: n = 256, 512, 1024), FP32.
// One warp computes one length-n DFT with no CTA barrier (four-step factorisation
// n = V x 32):
//   1. lane l holds x[l + 32 m], m < V; a V-point DFT over m in registers gives A_l(k1);
//   2. A_l(k1) is multiplied by W_n^{l k1} and transposed through a warp-private shared
//      buffer, so that the G = 32 / V lanes of group k1 hold the 32 values over l;
//   3. with l = la + G lb, a V-point DFT over lb in registers, the twiddle W_32^{la k2'}
//      and a G-point DFT across the group's lanes (shuffles) give
//      X[k1 + V k2' + V^2 k2''].
// The adjoint steps in reverse order (conjugate twiddles, decimation in time) map that
// layout back to lane l holding y[l + 32 m]: the unnormalised inverse DFT.  So the
// column pass multiplies by the symbol in the scrambled layout and the inverse row pass
// loads its coefficients straight into it.

// cos(2 pi j / 32) for 0 <= j <= 8: cos(k pi / 16), k = 0..8
__host__ __device__ constexpr double w32_octant(int j)
{
    return j == 0 ? 1.0
         : j == 1 ? 0.98078528040323044913
         : j == 2 ? 0.92387953251128675613
         : j == 3 ? 0.83146961230254523708
         : j == 4 ? 0.70710678118654752440
         : j == 5 ? 0.55557023301960222474
         : j == 6 ? 0.38268343236508977173
         : j == 7 ? 0.19509032201612826785
         : 0.0;
}
// cos and sin of 2 pi t / 32 for any integer t, by quadrant symmetry
__host__ __device__ constexpr float w32_cos(int t)
{
    return (t & 31) <= 8 ? (float)w32_octant(t & 31)
         : (t & 31) <= 16 ? (float)-w32_octant(16 - (t & 31))
         : (t & 31) <= 24 ? (float)-w32_octant((t & 31) - 16)
         : (float)w32_octant(32 - (t & 31));
}
__host__ __device__ constexpr float w32_sin(int t) { return w32_cos(t - 8); }

// d * exp(S 2 pi i t / 32) (t a compile-time constant after unrolling: the quarter turns
// are exact swaps and sign changes)
template <int S>
__device__ __forceinline__ float2 rot32(float2 d, int t)
{
    t &= 31;
    if (t == 0) return d;
    if (t == 8) return S > 0 ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
    if (t == 16) return make_float2(-d.x, -d.y);
    if (t == 24) return S > 0 ? make_float2(d.y, -d.x) : make_float2(-d.y, d.x);
    const float c = w32_cos(t), s = (float)S * w32_sin(t);
    return make_float2(d.x * c - d.y * s, d.x * s + d.y * c);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// W_n^{S t} from the table tw[t] = exp(-2 pi i t / n) (staged in shared memory)
template <int S>
__device__ __forceinline__ float2 tw_n(const float2 *tw, int t)
{
    float2 w = tw[t];
    if (S > 0) w.y = -w.y;
    return w;
}

// the twiddle table into shared memory, 16 bytes per thread and step
template <int N>
__device__ __forceinline__ void stage_tw(float2 *s_tw, const float2 *__restrict__ tw)
{
    const float4 *src = reinterpret_cast<const float4 *>(tw);
    float4 *dst = reinterpret_cast<float4 *>(s_tw);
    for (int t = threadIdx.x; t < N / 2; t += blockDim.x) dst[t] = __ldg(src + t);
}

template <int B> __host__ __device__ constexpr int brev(int i)
{
    int r = 0;
    for (int b = 0; b < B; ++b) r |= ((i >> b) & 1) << (B - 1 - b);
    return r;
}
template <int V> __host__ __device__ constexpr int ilog2c() { return V <= 1 ? 0 : 1 + ilog2c<V / 2>(); }

// V-point DFT with sign S in registers, decimation in frequency: natural order in,
// v[i] = X[brev(i)] out.
template <int V, int S>
__device__ __forceinline__ void dft_dif(float2 (&v)[V])
{
    constexpr int L = ilog2c<V>();
#pragma unroll
    for (int st = 0; st < L; ++st) {
        const int span = V >> (st + 1);
#pragma unroll
        for (int b = 0; b < V; b += 2 * span)
#pragma unroll
            for (int j = 0; j < span; ++j) {
                const float2 a = v[b + j], c = v[b + j + span];
                v[b + j] = make_float2(a.x + c.x, a.y + c.y);
                v[b + j + span] = rot32<S>(make_float2(a.x - c.x, a.y - c.y), j * (16 / span));
            }
    }
}

// Its adjoint up to the sign: decimation in time, v[i] = X[brev(i)] in, natural order out
// (dft_dit<V, +1> after dft_dif<V, -1> is V times the identity).
template <int V, int S>
__device__ __forceinline__ void dft_dit(float2 (&v)[V])
{
    constexpr int L = ilog2c<V>();
#pragma unroll
    for (int st = L - 1; st >= 0; --st) {
        const int span = V >> (st + 1);
#pragma unroll
        for (int b = 0; b < V; b += 2 * span)
#pragma unroll
            for (int j = 0; j < span; ++j) {
                const float2 a = v[b + j], c = rot32<S>(v[b + j + span], j * (16 / span));
                v[b + j] = make_float2(a.x + c.x, a.y + c.y);
                v[b + j + span] = make_float2(a.x - c.x, a.y - c.y);
            }
    }
}

__device__ __forceinline__ float2 shfl_xor2(float2 v, int d)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, d), __shfl_xor_sync(0xffffffffu, v.y, d));
}

// G-point DFT (sign S) across the lanes la = lane % G of a group, decimation in
// frequency: lane la ends with coefficient brev(la).
template <int V, int G, int S>
__device__ __forceinline__ void xlane_dif(float2 (&v)[V], int la)
{
#pragma unroll
    for (int d = G / 2; d >= 1; d >>= 1) {
        const bool bot = (la & d) != 0;
        const bool turn = bot && (la & (d - 1)) != 0;      // d = 2, la = 3: W_4^{S}
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const float2 p = shfl_xor2(v[i], d), x = v[i];
            float2 o = bot ? make_float2(p.x - x.x, p.y - x.y) : make_float2(x.x + p.x, x.y + p.y);
            if (turn) o = rot32<S>(o, 8);
            v[i] = o;
        }
    }
}

// Adjoint of xlane_dif (with S = +1 after a forward S = -1): stages in reverse order.
template <int V, int G, int S>
__device__ __forceinline__ void xlane_dit(float2 (&v)[V], int la)
{
#pragma unroll
    for (int d = 1; d < G; d <<= 1) {
        const bool bot = (la & d) != 0;
        const bool turn = bot && (la & (d - 1)) != 0;
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const float2 t = turn ? rot32<S>(v[i], 8) : v[i];
            const float2 p = shfl_xor2(t, d);
            v[i] = bot ? make_float2(p.x - t.x, p.y - t.y) : make_float2(t.x + p.x, t.y + p.y);
        }
    }
}

// frequency held by (lane, register i) after wfft_fwd
template <int V>
__device__ __forceinline__ int wfft_k(int lane, int i)
{
    constexpr int G = 32 / V;
    return lane / G + V * brev<ilog2c<V>()>(i) + V * V * brev<ilog2c<G>()>(lane % G);
}

// Forward (S = -1) or inverse (S = +1) length-32V DFT of one warp: v[m] = x[lane + 32 m]
// in, v[i] = X[wfft_k(lane, i)] out.  buf: (32 + G) V complex of this warp's shared memory.
template <int V, int S>
__device__ __forceinline__ void wfft_fwd(float2 (&v)[V], int lane, float2 *buf, const float2 *tw)
{
    constexpr int G = 32 / V, P = 32 + G, LB = ilog2c<V>();
    dft_dif<V, S>(v);
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const int k1 = brev<LB>(i);
        buf[k1 * P + lane] = k1 ? cmulf(v[i], tw_n<S>(tw, lane * k1)) : v[i];
    }
    __syncwarp();
    const int k1 = lane / G, la = lane % G;
#pragma unroll
    for (int lb = 0; lb < V; ++lb) v[lb] = buf[k1 * P + la + G * lb];
    __syncwarp();
    dft_dif<V, S>(v);
    if (G > 1 && la) {
#pragma unroll
        for (int i = 1; i < V; ++i) v[i] = cmulf(v[i], tw_n<S>(tw, la * brev<LB>(i) * V));
    }
    xlane_dif<V, G, S>(v, la);
}

// The adjoint steps of wfft_fwd<V, -S>: v[i] = X[wfft_k(lane, i)] in, v[m] = y[lane + 32 m]
// out, y[j] = sum_k X[k] exp(S 2 pi i j k / n) (S = +1: the unnormalised inverse DFT).
template <int V, int S>
__device__ __forceinline__ void wfft_adj(float2 (&v)[V], int lane, float2 *buf, const float2 *tw)
{
    constexpr int G = 32 / V, P = 32 + G, LB = ilog2c<V>();
    const int k1 = lane / G, la = lane % G;
    xlane_dit<V, G, S>(v, la);
    if (G > 1 && la) {
#pragma unroll
        for (int i = 1; i < V; ++i) v[i] = cmulf(v[i], tw_n<S>(tw, la * brev<LB>(i) * V));
    }
    dft_dit<V, S>(v);
#pragma unroll
    for (int lb = 0; lb < V; ++lb) buf[k1 * P + la + G * lb] = v[lb];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const int kk = brev<LB>(i);
        const float2 x = buf[kk * P + lane];
        v[i] = kk ? cmulf(x, tw_n<S>(tw, lane * kk)) : x;
    }
    __syncwarp();
    dft_dit<V, S>(v);
}

#ifndef CTR_WFFT_COL_WARPS
#define CTR_WFFT_COL_WARPS 4
#endif
#ifndef CTR_WFFT_INV_WARPS
#define CTR_WFFT_INV_WARPS 2
#endif
// adjacent columns per CTA of the column pass (they share L1 sectors; at V = 32 at most 4,
// the static shared-memory limit) and row pairs per CTA of the inverse row pass
template <int V> constexpr int wfft_col_warps() { return V >= 32 && CTR_WFFT_COL_WARPS > 4 ? 4 : CTR_WFFT_COL_WARPS; }
constexpr int WFFT_INV_WARPS = CTR_WFFT_INV_WARPS;

// Forward row pass of the real-input form, one row pair per CTA: the CTA's 256 threads
// form the real inputs of rows 2b and 2b + 1 (the fold of the backprojection's partial
// planes and the step-A epilogue, or a real image) into shared memory with many loads in
// flight, then one warp transforms z = x_a + i x_b and writes X_a(k), X_b(k), k <= n/2.
template <int V>
__global__ void __launch_bounds__(FFT_THREADS)
k_wfft_rows_fwd_packed(RowsInput<float> src, float2 *cbuf, const float2 *__restrict__ tw)
{
    constexpr int n = 32 * V, H = n / 2 + 1, G = 32 / V;
    __shared__ __align__(16) float s_in[2 * n];
    __shared__ __align__(16) float2 s_buf[(32 + G) * V];
    __shared__ __align__(16) float2 s_tw[n];
    const int ra = 2 * blockIdx.x;
    pdl_wait();
    pdl_trigger();
    stage_tw<n>(s_tw, tw);
    if (src.part && src.orbit) {
        // the fold of the partial planes four columns at a time (16-byte loads; each column's
        // sum in the order of orbit_fold), then the step-A epilogue per pixel
        for (int e4 = threadIdx.x; e4 < n / 2; e4 += blockDim.x) {
            const int row = ra + (4 * e4 >= n ? 1 : 0), col = (4 * e4) & (n - 1);
            const float4 acc = orbit_fold4(src.part, src.groups, n, row, col);
            float *dst = s_in + 4 * e4;
            dst[0] = bp_epilogue_value(src.epi, n, row, col, acc.x);
            dst[1] = bp_epilogue_value(src.epi, n, row, col + 1, acc.y);
            dst[2] = bp_epilogue_value(src.epi, n, row, col + 2, acc.z);
            dst[3] = bp_epilogue_value(src.epi, n, row, col + 3, acc.w);
        }
    } else {
        staged_copy(2 * n, [&](int e) { return rows_input_value(src, n, ra + (e >= n ? 1 : 0), e & (n - 1)); },
                    [&](int e, float x) { s_in[e] = x; });
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    float2 v[V];
#pragma unroll
    for (int m = 0; m < V; ++m) v[m] = make_float2(s_in[lane + 32 * m], s_in[n + lane + 32 * m]);
    wfft_fwd<V, -1>(v, lane, s_buf, s_tw);
#pragma unroll
    for (int i = 0; i < V; ++i) s_buf[wfft_k<V>(lane, i)] = v[i];     // natural order (n <= (32 + G) V)
    __syncwarp();
    float2 *xa_row = cbuf + (size_t)ra * H, *xb_row = xa_row + H;
    for (int k = lane; k < H; k += 32) {
        const float2 z = s_buf[k], zm = s_buf[(n - k) & (n - 1)];
        xa_row[k] = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
        xb_row[k] = make_float2(0.5f * (z.y + zm.y), 0.5f * (zm.x - z.x));
    }
}

// Column pass of the real-input form: one warp per stored column c < n/2 + 1: forward
// DFT, times the real symbol sym[k][c] in the scrambled layout, inverse DFT.
template <int V>
__global__ void __launch_bounds__(32 * wfft_col_warps<V>())
k_wfft_cols_packed(float2 *cbuf, const float *__restrict__ sym, const float2 *__restrict__ tw)
{
    constexpr int n = 32 * V, H = n / 2 + 1, G = 32 / V;
    constexpr int CW = wfft_col_warps<V>();
    __shared__ __align__(16) float2 s_buf[CW][(32 + G) * V];
    __shared__ __align__(16) float2 s_tw[n];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * CW + w;
    const bool live = c < H;                             // warp-uniform
    pdl_wait();
    pdl_trigger();
    float2 v[V];
    float sy[V];                                         // the symbol, fetched with the data
    if (live) {
#pragma unroll
        for (int m = 0; m < V; ++m) v[m] = cbuf[(size_t)(lane + 32 * m) * H + c];
#pragma unroll
        for (int i = 0; i < V; ++i) sy[i] = __ldg(sym + (size_t)wfft_k<V>(lane, i) * n + c);
    }
    stage_tw<n>(s_tw, tw);
    __syncthreads();
    if (!live) return;
    wfft_fwd<V, -1>(v, lane, s_buf[w], s_tw);
#pragma unroll
    for (int i = 0; i < V; ++i) {
        v[i].x *= sy[i];
        v[i].y *= sy[i];
    }
    wfft_adj<V, +1>(v, lane, s_buf[w], s_tw);
#pragma unroll
    for (int m = 0; m < V; ++m) cbuf[(size_t)(lane + 32 * m) * H + c] = v[m];
}

// Inverse row pass of the real-input form: one warp per row pair, the coefficients loaded
// straight into the scrambled layout (X(k) = conj X(n - k) beyond n/2), Z = X_a + i X_b
// inverted, real part -> row 2c, imaginary part -> row 2c + 1, with the epilogue of
// fft_rows_inv_packed_body (mode 0: out = v; mode 1: out += v; dout = v; bfloat16 copies;
// transposed copies written as (row 2c, row 2c + 1) pairs).
template <int V>
__global__ void __launch_bounds__(32 * WFFT_INV_WARPS)
k_wfft_rows_inv_packed(const float2 *__restrict__ cbuf, const float2 *__restrict__ tw, float *out, int mode,
                       float *outT, float *dout, __nv_bfloat16 *outh, __nv_bfloat16 *outTh)
{
    constexpr int n = 32 * V, H = n / 2 + 1, G = 32 / V;
    __shared__ __align__(16) float2 s_buf[WFFT_INV_WARPS][(32 + G) * V];
    __shared__ __align__(16) float2 s_tw[n];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ra = 2 * (blockIdx.x * WFFT_INV_WARPS + w);     // < n: the grid covers n / 2 row pairs exactly
    pdl_wait();
    pdl_trigger();
    stage_tw<n>(s_tw, tw);
    const float2 *xa_row = cbuf + (size_t)ra * H, *xb_row = xa_row + H;
    float2 v[V];
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const int k = wfft_k<V>(lane, i);
        const bool lo = k <= n / 2;
        const int kk = lo ? k : n - k;
        float2 xa = xa_row[kk], xb = xb_row[kk];
        if (!lo) {
            xa.y = -xa.y;
            xb.y = -xb.y;
        }
        v[i] = make_float2(xa.x - xb.y, xa.y + xb.x);
    }
    float pa[V], pb[V];
    const size_t ga = (size_t)ra * n, gb = ga + n;
#pragma unroll
    for (int m = 0; m < V; ++m) {
        pa[m] = mode == 1 ? out[ga + lane + 32 * m] : 0.f;
        pb[m] = mode == 1 ? out[gb + lane + 32 * m] : 0.f;
    }
    __syncthreads();
    wfft_adj<V, +1>(v, lane, s_buf[w], s_tw);
#pragma unroll
    for (int m = 0; m < V; ++m) {
        const int j = lane + 32 * m;
        const float va = v[m].x, vb = v[m].y;
        if (dout) {
            dout[ga + j] = va;
            dout[gb + j] = vb;
        }
        const float oa = va + pa[m], ob = vb + pb[m];
        out[ga + j] = oa;
        out[gb + j] = ob;
        if (outh) {
            outh[ga + j] = __float2bfloat16_rn(oa);
            outh[gb + j] = __float2bfloat16_rn(ob);
        }
        if (outT) *reinterpret_cast<float2 *>(outT + (size_t)j * n + ra) = make_float2(oa, ob);
        if (outTh) *reinterpret_cast<__nv_bfloat162 *>(outTh + (size_t)j * n + ra) = __floats2bfloat162_rn(oa, ob);
    }
}

// The warp-level form covers FP32 plans with n = 256, 512 or 1024.
int wfft_v(const ctr_plan *p)
{
    if (p->esize != 4) return 0;
    return p->n == 256 ? 8 : p->n == 512 ? 16 : p->n == 1024 ? 32 : 0;
}

template <int V>
void launch_wfft_packed(bool pdl, const RowsInput<float> &src, float2 *cb, const float *sym, const float2 *tw,
                        float *out, int mode, float *outT, float *dout, __nv_bfloat16 *outh, __nv_bfloat16 *outTh,
                        cudaStream_t s)
{
    constexpr int n = 32 * V, H = n / 2 + 1;
    launch_pdl(pdl, k_wfft_rows_fwd_packed<V>, dim3(n / 2), dim3(FFT_THREADS), 0, s, src, cb, tw);
    constexpr int CW = wfft_col_warps<V>();
    launch_pdl(pdl, k_wfft_cols_packed<V>, dim3((H + CW - 1) / CW), dim3(32 * CW), 0,
               s, cb, sym, tw);
    launch_pdl(pdl, k_wfft_rows_inv_packed<V>, dim3(n / (2 * WFFT_INV_WARPS)), dim3(32 * WFFT_INV_WARPS), 0, s,
               (const float2 *)cb, tw, out, mode, outT, dout, outh, outTh);
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
    RowsInput<float> src{};
    if (d.orbit || d.bp_groups > 1) {             // the backprojection left partial images
        src.part = d.bp_part;
        src.groups = d.bp_groups;
        src.orbit = d.orbit;
        src.epi = d.bpe;
    }
    if (d.packed) fft_rows_fwd_packed_body<float>(src, d.cbuf, d.n, d.prp, d.fp, d.tw, blockIdx.x - prefix[s]);
    else fft_rows_fwd_body<float>(src, d.cbuf, d.n, d.rpc, d.fp, d.tw, blockIdx.x - prefix[s]);
}

__global__ void __launch_bounds__(FFT_THREADS)
k_fft_cols_batch(const SliceDesc *__restrict__ sd, const int *__restrict__ prefix, int ns)
{
    const int s = find_slice_fft(prefix, ns, blockIdx.x);
    const SliceDesc &d = sd[s];
    if (d.packed) fft_cols_body<float>(d.cbuf, d.sym, d.n, d.pcw, d.fp, d.tw, blockIdx.x - prefix[s], 0, d.n / 2 + 1,
                                       d.n / 2 + 1);
    else fft_cols_body<float>(d.cbuf, d.sym, d.n, d.cw, d.fp, d.tw, blockIdx.x - prefix[s], d.twist);
}

__global__ void __launch_bounds__(FFT_THREADS)
k_fft_rows_inv_batch(const SliceDesc *__restrict__ sd, const int *__restrict__ prefix, int ns)
{
    const int s = find_slice_fft(prefix, ns, blockIdx.x);
    const SliceDesc &d = sd[s];
    if (d.packed)
        fft_rows_inv_packed_body<float>(d.cbuf, d.n, d.prp, d.fp, d.tw, d.u, 1, d.orbit ? nullptr : d.uT, nullptr,
                                        nullptr, nullptr, blockIdx.x - prefix[s]);
    else
        fft_rows_inv_body<float>(d.cbuf, d.n, d.rpc, d.fp, d.tw, d.u, 1, d.orbit ? nullptr : d.uT, nullptr, nullptr,
                                 nullptr, blockIdx.x - prefix[s]);
}

// Preconditioner symbols (Alg. 4, Sec. 4.3.1), with 1/n^2 of the inverse DFT:
//   sym  = ||xi||_eps / (sigma^2 c + (sigma tau)^2 L ||xi||_eps) / n^2
//   symh = sqrt(||xi||_eps) / n^2
template <typename T>
__global__ void k_symbols(T *sym, T *symh, int n, double sigma, double tau, double c, double eps, int nonneg,
                          int kind, double inv_h2, const T *__restrict__ s_arr)
{
    const size_t total = (size_t)n * n;
    const double pi = 3.14159265358979323846;
    const double inv_n2 = 1.0 / ((double)n * (double)n);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = pix_i(e, n), j = pix_j(e, n);
        const int ii = (2 * i < n) ? i : i - n;    // wrapped signed index (Nyquist sign irrelevant)
        const int jj = (2 * j < n) ? j : j - n;
        const double xi = 2.0 * pi * ii / n, xj = 2.0 * pi * jj / n;
        const double nrm = sqrt(xi * xi + xj * xj + eps * eps);
        const double si = sin(pi * i / n), sj = sin(pi * j / n);
        const double L = 4.0 * si * si + 4.0 * sj * sj;
        const double st2 = (sigma * tau) * (sigma * tau), id1 = nonneg ? 1.0 : 0.0;
        if (kind == 3) {
            // Richardson: M = (sigma^2 c + (sigma tau)^2 8 / h^2) id (+ id), S = id
            sym[e] = (T)(inv_n2 / (id1 + sigma * sigma * c + st2 * 8.0 * inv_h2));
            if (symh) symh[e] = (T)inv_n2;
            continue;
        }
        if (kind == 1 || kind == 2) {
            // M = sigma^2 c S + (sigma tau)^2 Lap (+ id), S the convolution (kind 1, 2-D DFT s)
            // or the circulant (kind 2, 1-D DFT s of the flattened image, position e = flat
            // frequency k) with Lap = -Delta_p resp. the circulant of -Delta_h, whose
            // 1-D DFT is (4 - 2 cos(2 pi k / n^2) - 2 cos(2 pi k / n)) / h^2
            const double sv = (double)s_arr[e];
            double Lk = L;
            if (kind == 2) {
                const double nn2 = (double)n * (double)n;
                Lk = (4.0 - 2.0 * cospi(2.0 * (double)e / nn2) - 2.0 * cospi(2.0 * (double)j / n)) * inv_h2;
            }
            sym[e] = (T)(inv_n2 / (id1 + sigma * sigma * c * sv + st2 * Lk));
            if (symh) symh[e] = (T)(inv_n2 / sqrt(sv));
            continue;
        }
        const double id = nonneg ? nrm : 0.0;   // Alg. 5: M = id + c sigma^2 F^{-1}(1/||xi||)F - (sigma tau)^2 Delta
        sym[e] = (T)(nrm / (id + sigma * sigma * c + (sigma * tau) * (sigma * tau) * L * nrm) * inv_n2);
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

int rows_per_cta(const ctr_plan *p) { return fft_rows_per_cta(p->n); }
int cols_per_cta(const ctr_plan *p) { return fft_cols_per_cta(p->n, p->esize); }
// real-input form: an even number of rows per CTA (pairs share a complex FFT), about the
// same points per CTA as the complex form; columns: half as many per CTA (half remain)
#ifndef CTR_PACK_ROWS_MUL
#define CTR_PACK_ROWS_MUL 1
#endif
#ifndef CTR_PACK_COLS_MUL
#define CTR_PACK_COLS_MUL 1
#endif
int packed_rows_per_cta(const ctr_plan *p)
{
    return 2 * CTR_PACK_ROWS_MUL * (fft_rows_per_cta(p->n) > 1 ? fft_rows_per_cta(p->n) / 2 : 1);
}
int packed_cols_per_cta(const ctr_plan *p)
{
    int c = CTR_PACK_COLS_MUL * (cols_per_cta(p) > 1 ? cols_per_cta(p) / 2 : 1);
    while (c > 1 && 2 * (size_t)c * (p->n + 1) * 2 * p->esize > 160 * 1024) c /= 2;
    return c;
}
size_t packed_rows_smem(const ctr_plan *p) { return (2 * (size_t)(packed_rows_per_cta(p) / 2) * p->n + p->n) * 2 * p->esize; }
size_t packed_cols_smem(const ctr_plan *p) { return (2 * (size_t)packed_cols_per_cta(p) * (p->n + 1) + p->n) * 2 * p->esize; }

}  // namespace

bool wfft_supported(const ctr_plan *p) { return wfft_v(p) != 0; }
int fft_packed_rows_per_cta(const ctr_plan *p) { return packed_rows_per_cta(p); }
int fft_packed_cols_per_cta(const ctr_plan *p) { return packed_cols_per_cta(p); }
size_t fft_packed_smem(const ctr_plan *p, int which) { return which == 0 ? packed_rows_smem(p) : packed_cols_smem(p); }

size_t fft_smem_bytes(const ctr_plan *p, int which)
{
    return which == 0 ? fft_rows_smem(p->n, p->esize) : fft_cols_smem(p->n, p->esize);
}

template <typename T>
ctr_status launch_circulant(const ctr_plan *p, const T *in_real, bool in_is_cbuf, const T *sym, T *out, int mode,
                            T *outT, T *dout, cudaStream_t s, __nv_bfloat16 *outh, __nv_bfloat16 *outTh,
                            const BackprojEpi<T> *bp_in)
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
    RowsInput<T> src{};
    if (bp_in) {
        src.orbit = sizeof(T) == 4 && p->orbit;
        src.part = (const T *)(src.orbit ? p->obp_part : p->bp_part);
        src.groups = src.orbit ? p->obp_groups : p->bp_groups;
        src.epi = *bp_in;
    } else if (!in_is_cbuf) {
        src.in_real = in_real;
    }
    // Real-input form: real image in, real image out and a real even symbol (every kind
    // but the circulant one, whose 1-D transform is not the 2-D DFT); its packed rows
    // would overwrite unread input rows if the input were cbuf itself.
    if (p->precond_kind != 2 && (bp_in || !in_is_cbuf)) {
        if constexpr (sizeof(T) == 4) {
            const int V = p->fft_form == 0 ? wfft_v(p) : 0;
            if (V) {
                p->launches += 2;
                const bool pdl = p->pdl != 0;
                if (V == 8) launch_wfft_packed<8>(pdl, src, cb, sym, tw, out, mode, outT, dout, outh, outTh, s);
                else if (V == 16) launch_wfft_packed<16>(pdl, src, cb, sym, tw, out, mode, outT, dout, outh, outTh, s);
                else launch_wfft_packed<32>(pdl, src, cb, sym, tw, out, mode, outT, dout, outh, outTh, s);
                CTR_CHECK_LAUNCH("k_wfft_packed");
                return CTR_OK;
            }
        }
        const int prp = packed_rows_per_cta(p), pcw = packed_cols_per_cta(p);
        const int pgr = (n + prp - 1) / prp, pgc = (n / 2 + 1 + pcw - 1) / pcw;
        const size_t psr = packed_rows_smem(p), psc = packed_cols_smem(p);
        k_fft_rows_fwd_packed<T><<<pgr, FFT_THREADS, psr, s>>>(src, cb, n, prp, fp, tw);
        CTR_CHECK_LAUNCH("k_fft_rows_fwd_packed");
        p->launches++;
        k_fft_cols_packed<T><<<pgc, FFT_THREADS, psc, s>>>(cb, sym, n, pcw, fp, tw);
        CTR_CHECK_LAUNCH("k_fft_cols_packed");
        p->launches++;
        k_fft_rows_inv_packed<T><<<pgr, FFT_THREADS, psr, s>>>(cb, n, prp, fp, tw, out, mode, outT, dout, outh,
                                                               outTh);
        CTR_CHECK_LAUNCH("k_fft_rows_inv_packed");
        return CTR_OK;
    }
    k_fft_rows_fwd<T><<<gr, FFT_THREADS, smr, s>>>(src, cb, n, rpc, fp, tw);
    CTR_CHECK_LAUNCH("k_fft_rows_fwd");
    p->launches++;
    k_fft_cols<T><<<gc, FFT_THREADS, smc, s>>>(cb, sym, n, cw, fp, tw, p->precond_kind == 2 ? 1 : 0);
    CTR_CHECK_LAUNCH("k_fft_cols");
    p->launches++;
    k_fft_rows_inv<T><<<gr, FFT_THREADS, smr, s>>>(cb, n, rpc, fp, tw, out, mode, outT, dout, outh, outTh);
    CTR_CHECK_LAUNCH("k_fft_rows_inv");
    return CTR_OK;
}

// cbuf = F2(in_real), the plain 2-D forward DFT (row pass, then the column pass alone).
template <typename T>
ctr_status launch_fft2_forward(const ctr_plan *p, const T *in_real, cudaStream_t s, bool twist)
{
    using T2 = typename C2<T>::type;
    const int n = p->n;
    const FftPasses fp = make_passes(p);
    const T2 *tw = reinterpret_cast<const T2 *>(p->d_twiddle);
    T2 *cb = reinterpret_cast<T2 *>(p->cbuf);
    const int rpc = rows_per_cta(p), cw = cols_per_cta(p);
    RowsInput<T> src{};
    src.in_real = in_real;
    p->launches++;
    k_fft_rows_fwd<T><<<(n + rpc - 1) / rpc, FFT_THREADS, fft_smem_bytes(p, 0), s>>>(src, cb, n, rpc, fp, tw);
    CTR_CHECK_LAUNCH("k_fft_rows_fwd");
    p->launches++;
    k_fft_cols<T><<<(n + cw - 1) / cw, FFT_THREADS, fft_smem_bytes(p, 1), s>>>(cb, nullptr, n, cw, fp, tw,
                                                                              twist ? 1 : 0);
    CTR_CHECK_LAUNCH("k_fft_cols");
    return CTR_OK;
}
template ctr_status launch_fft2_forward<float>(const ctr_plan *, const float *, cudaStream_t, bool);
template ctr_status launch_fft2_forward<double>(const ctr_plan *, const double *, cudaStream_t, bool);

// Detector-axis ramp filter (Sec. 2): per view, the bins zero-padded to L, forward FFT,
// times the real multiplier H (the DFT of the Ram-Lak kernel wrapped onto L points, with
// ds / L folded in), inverse FFT, the first M outputs times outscale: the linear
// convolution of each view with the kernel.
template <typename T>
__global__ void __launch_bounds__(FFT_THREADS)
k_ramp_filter(const T *__restrict__ g, int N, int M, int L, int rpc, FftPasses fp,
              const typename C2<T>::type *__restrict__ tw, const T *__restrict__ H, T outscale, T *y,
              __nv_bfloat16 *yh)
{
    using T2 = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *a = reinterpret_cast<T2 *>(smem_raw);
    T2 *b = a + (size_t)rpc * L;
    T2 *stw = b + (size_t)rpc * L;
    stage_twiddles(stw, tw, L);
    const int l0 = blockIdx.x * rpc;
    const int cnt = min(rpc, N - l0);
    for (int e = threadIdx.x; e < cnt * L; e += blockDim.x) {
        const int r = e / L, k = e - r * L;
        T2 v;
        v.x = k < M ? g[(size_t)(l0 + r) * M + k] : T(0);
        v.y = T(0);
        a[e] = v;
    }
    __syncthreads();
    T2 *res = fft_smem<T>(a, b, L, cnt, L, fp, -1, stw);
    for (int e = threadIdx.x; e < cnt * L; e += blockDim.x) {
        const T m = H[e % L];
        res[e].x *= m;
        res[e].y *= m;
    }
    __syncthreads();
    T2 *res2 = fft_smem<T>(res, res == a ? b : a, L, cnt, L, fp, +1, stw);
    for (int e = threadIdx.x; e < cnt * M; e += blockDim.x) {
        const int r = e / M, k = e - r * M;
        const T v = res2[(size_t)r * L + k].x * outscale;
        const size_t o = (size_t)(l0 + r) * M + k;
        if (yh) yh[o] = __float2bfloat16_rn((float)v);
        else y[o] = v;
    }
}

size_t ramp_smem(int L, size_t esize) { return (2 * (size_t)fft_rows_per_cta(L) * L + L) * 2 * esize; }

// The ramp tables: twiddles e^{-2 pi i t / L} and H(t) = (ds / L) sum_m k(m) cos(2 pi m t / L)
// with the Ram-Lak kernel k(0) = 1/(4 ds^2), k(m) = -1/(pi^2 m^2 ds^2) for odd |m| < M.
template <typename T>
ctr_status prepare_ramp(ctr_plan *p)
{
    if (p->ramp_ready) return CTR_OK;
    const int L = p->ramp_L, M = p->M;
    if (ramp_smem(L, sizeof(T)) > 227 * 1024)
        return fail(CTR_EUNSUPPORTED, "detector too long for the shared-memory ramp filter in this precision "
                                      "(one view of 2M - 1 padded points must fit one CTA)");
    const double pi = 3.14159265358979323846, ds = p->ds;
    std::vector<T> tw(2 * (size_t)L), H(L);
    for (int t = 0; t < L; ++t) {
        tw[2 * t] = (T)cos(2.0 * pi * t / L);
        tw[2 * t + 1] = (T)(-sin(2.0 * pi * t / L));
    }
    for (int t = 0; t < L; ++t) {
        double acc = 1.0 / (4.0 * ds * ds);
        for (int m = 1; m < M; m += 2) {
            const long long r = ((long long)m * t) % L;
            acc += 2.0 * (-1.0 / (pi * pi * (double)m * m * ds * ds)) * cos(2.0 * pi * (double)r / L);
        }
        H[t] = (T)(acc * ds / L);
    }
    CTR_CUDA(cudaMemcpy(p->d_ramp_tw, tw.data(), sizeof(T) * tw.size(), cudaMemcpyHostToDevice));
    CTR_CUDA(cudaMemcpy(p->d_ramp_H, H.data(), sizeof(T) * H.size(), cudaMemcpyHostToDevice));
    ctr_status st = raise_smem_limit(k_ramp_filter<T>, ramp_smem(L, sizeof(T)));
    if (st != CTR_OK) return st;
    p->ramp_ready = true;
    return CTR_OK;
}

template <typename T>
ctr_status launch_ramp(ctr_plan *p, const T *g, T *y, __nv_bfloat16 *yh, double outscale, cudaStream_t s)
{
    ctr_status st = prepare_ramp<T>(p);
    if (st != CTR_OK) return st;
    FftPasses fp;
    fp.count = (int)p->ramp_radices.size();
    for (int i = 0; i < fp.count && i < MAX_PASSES; ++i) fp.radix[i] = p->ramp_radices[i];
    const int L = p->ramp_L, rpc = fft_rows_per_cta(L);
    p->launches++;
    k_ramp_filter<T><<<(p->N + rpc - 1) / rpc, FFT_THREADS, ramp_smem(L, sizeof(T)), s>>>(
        g, p->N, p->M, L, rpc, fp, reinterpret_cast<const typename C2<T>::type *>(p->d_ramp_tw),
        (const T *)p->d_ramp_H, (T)outscale, y, yh);
    CTR_CHECK_LAUNCH("k_ramp_filter");
    return CTR_OK;
}
template ctr_status launch_ramp<float>(ctr_plan *, const float *, float *, __nv_bfloat16 *, double, cudaStream_t);
template ctr_status launch_ramp<double>(ctr_plan *, const double *, double *, __nv_bfloat16 *, double, cudaStream_t);

template <typename T>
ctr_status configure_fft(const ctr_plan *p)
{
    const size_t smr = fft_smem_bytes(p, 0), smc = fft_smem_bytes(p, 1);
    ctr_status st = raise_smem_limit(k_fft_rows_fwd<T>, smr);
    if (st == CTR_OK) st = raise_smem_limit(k_fft_rows_inv<T>, smr);
    if (st == CTR_OK) st = raise_smem_limit(k_fft_cols<T>, smc);
    if (st == CTR_OK) st = raise_smem_limit(k_fft_rows_fwd_packed<T>, packed_rows_smem(p));
    if (st == CTR_OK) st = raise_smem_limit(k_fft_rows_inv_packed<T>, packed_rows_smem(p));
    if (st == CTR_OK) st = raise_smem_limit(k_fft_cols_packed<T>, packed_cols_smem(p));
    return st;
}

template <typename T>
ctr_status launch_symbols(const ctr_plan *p, double sigma, double tau, double c, double eps, cudaStream_t s,
                          bool nonneg)
{
    // the symbols of the last call are still in place if nothing they depend on changed
    const double key[SYM_KEY_LEN] = {sigma, tau, c, eps, nonneg ? 1.0 : 0.0, (double)p->precond_kind,
                                     (double)p->pk_kind, 1.0 / (p->h * p->h)};
    if (p->sym_valid && std::memcmp(key, p->sym_key, sizeof(key)) == 0) return CTR_OK;
    const size_t total = (size_t)p->n * p->n;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    p->launches++;
    std::memcpy(p->sym_key, key, sizeof(key));
    p->sym_valid = true;
    k_symbols<T><<<blocks, 256, 0, s>>>((T *)p->sym, (T *)p->symh, p->n, sigma, tau, c, eps, nonneg ? 1 : 0,
                                        p->precond_kind, 1.0 / (p->h * p->h), (const T *)p->pk_s);
    CTR_CHECK_LAUNCH("k_symbols");
    return CTR_OK;
}

template ctr_status launch_circulant<float>(const ctr_plan *, const float *, bool, const float *, float *, int, float *,
                                           float *, cudaStream_t, __nv_bfloat16 *, __nv_bfloat16 *,
                                           const BackprojEpi<float> *);
template ctr_status launch_circulant<double>(const ctr_plan *, const double *, bool, const double *, double *, int,
                                            double *, double *, cudaStream_t, __nv_bfloat16 *, __nv_bfloat16 *,
                                            const BackprojEpi<double> *);
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

// Work split of the FFT passes: about 1024 points per CTA of 128 threads, so that an
// n = 512 image gives 256 CTAs per pass.
// Shared memory of the passes: two ping-pong buffers plus the twiddle table.
size_t fft_rows_smem(int n, size_t esize)
{
    return (2 * (size_t)fft_rows_per_cta(n) * n + n) * 2 * esize;
}
size_t fft_cols_smem(int n, size_t esize)
{
    return (2 * (size_t)fft_cols_per_cta(n, esize) * (n + 1) + n) * 2 * esize;
}

int fft_rows_per_cta(int n)
{
    const int r = CTR_FFT_POINTS / n;
    return r < 1 ? 1 : (r > 16 ? 16 : r);
}

int fft_cols_per_cta(int n, size_t esize)
{
    int cw = CTR_FFT_POINTS / n;
    cw = cw < 1 ? 1 : (cw > 8 ? 8 : cw);
    while (cw > 1 && 2 * (size_t)cw * (n + 1) * 2 * esize > 160 * 1024) cw /= 2;
    return cw;
}

template ctr_status configure_fft<float>(const ctr_plan *);
template ctr_status configure_fft<double>(const ctr_plan *);
template ctr_status launch_symbols<float>(const ctr_plan *, double, double, double, double, cudaStream_t, bool);
template ctr_status launch_symbols<double>(const ctr_plan *, double, double, double, double, cudaStream_t, bool);

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
    // n <= 1024: rows_per_cta * n <= 1024 and cols_per_cta * (n + 1) <= 1024 + 8 points, plus
    // the twiddle table
    const int smax = (2 * (1024 + 8) + STATIC_MAX_N) * (int)sizeof(float2);
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
        std::vector<int> rad;
        if (fft_radices(n, rad) != CTR_OK)
            return fail(CTR_EUNSUPPORTED, "precond_apply_static: n must be of the form 2^a 3^b");
        fp.count = (int)rad.size();
        for (int i = 0; i < fp.count; ++i) fp.radix[i] = rad[i];
    }
    int dev = -1;
    CTR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= STATIC_MAX_DEVICES) return fail(CTR_EUNSUPPORTED, "precond_apply_static: device index too large");
    // both buffers must be device (or managed) memory of the current device; the
    // attribute query allocates nothing
    for (const void *p : {(const void *)y_dev, (const void *)x_dev}) {
        cudaPointerAttributes attr{};
        cudaError_t pe = cudaPointerGetAttributes(&attr, p);
        if (pe != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(CTR_EINVAL, "precond_apply_static: a buffer is not a CUDA pointer");
        }
        if ((attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) || attr.device != dev)
            return fail(CTR_EINVAL, "precond_apply_static: y_dev and x_dev must be device memory of the current "
                                    "device (cuda:" + std::to_string(dev) + ")");
    }
    ctr_status st = static_setup(dev);
    if (st != CTR_OK) return st;
    const StaticScratch &s = g_scratch[dev];
    cudaStream_t str = (cudaStream_t)stream;
    // the same three FFT passes as precond_apply, with every scratch in the static arrays
    k_static_twiddles<<<(n + 255) / 256, 256, 0, str>>>(s.tw, n);
    const size_t nn = (size_t)n * n;
    int blocks = (int)((nn + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_symbols<float><<<blocks, 256, 0, str>>>(s.sym, nullptr, n, sigma, tau, c, eps, 0, 0, 1.0, nullptr);
    const int rpc = fft_rows_per_cta(n), cw = fft_cols_per_cta(n, sizeof(float));
    const size_t smr = fft_rows_smem(n, sizeof(float)), smc = fft_cols_smem(n, sizeof(float));
    const int gr = (n + rpc - 1) / rpc, gc = (n + cw - 1) / cw;
    RowsInput<float> src{};
    src.in_real = y_dev;
    k_fft_rows_fwd<float><<<gr, FFT_THREADS, smr, str>>>(src, s.cbuf, n, rpc, fp, s.tw);
    k_fft_cols<float><<<gc, FFT_THREADS, smc, str>>>(s.cbuf, s.sym, n, cw, fp, s.tw, 0);
    k_fft_rows_inv<float><<<gr, FFT_THREADS, smr, str>>>(s.cbuf, n, rpc, fp, s.tw, x_dev, 0, nullptr, nullptr,
                                                         nullptr, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "precond_apply_static launch");
    return CTR_OK;
}
