// The discrete Radon transform R_h and its adjoint R_h^* (linear backprojection)
// of Sec. 3.1, as an exact transpose pair of gather kernels for sm_103a.
//
//  * R_h^* (pixel-driven): a CTA owns a 32 x 32 tile of pixels and one group of
//    angles; per chunk of 32 angles it stages, for every angle, the tile's
//    detector footprint into shared memory as interpolation-ready pairs, then each
//    thread walks its 8 pixels' exact fixed-point detector coordinate P and spends
//    one shared-memory load and one FMA per (pixel, angle).  With several angle
//    groups the groups' partial images are summed by a small epilogue kernel
//    (enough CTAs to fill 152 SMs at n = 512).  No atomics.
//  * R_h (ray-driven): one lane per detector interval [k, k+1) of one angle
//    marches across the image rows, tracking exactly (integer arithmetic) the
//    first pixel whose coordinate falls in its interval; it accumulates
//    sum u and sum frac*u over the pixels of its interval, and the two neighbouring
//    intervals' sums are combined with one warp shuffle:
//        g_k = sum_{floor p = k} (1 - frac) u  +  sum_{floor p = k-1} frac u.
//    A CTA takes 4 adjacent angles (one warp each) over 31 bins; the rows on which
//    every lane of a warp stays inside the image run without bounds checks.
//    No atomics; each output bin is written once.
// Both kernels derive each weight from the same integer P (see ctr_internal.cuh),
// so they are transposes of one matrix, bit for bit in the weights.
#include <algorithm>
#include <type_traits>

#include "ctr_internal.cuh"

namespace ctr {

namespace {

// CTA barrier of a stage body.  NAMED: the body runs on the first 128 threads of a larger
// CTA (the persistent batched iteration) and synchronises them with named barrier 1.
template <bool NAMED>
__device__ __forceinline__ void body_sync()
{
    if constexpr (NAMED) asm volatile("bar.sync 1, 128;" ::: "memory");
    else __syncthreads();
}

#ifndef CTR_BP_TY
#define CTR_BP_TY 4
#endif
#ifndef CTR_BP_R
#define CTR_BP_R 8
#endif
#ifndef CTR_BP_ACH
#define CTR_BP_ACH 32
#endif
constexpr int BP_TJ = 32;          // tile width along j (one warp)
constexpr int BP_TY = CTR_BP_TY;   // warps per CTA
constexpr int BP_R = CTR_BP_R;     // pixels per thread (rows i0 + ty + BP_TY r)
constexpr int BP_TI = BP_TY * BP_R;
constexpr int BP_ACH = CTR_BP_ACH; // angles per staged chunk

template <typename T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

// operand loads: FP32/FP64 as stored, bfloat16 widened to FP32
__device__ __forceinline__ float ldv(const float *p) { return *p; }
__device__ __forceinline__ double ldv(const double *p) { return *p; }
__device__ __forceinline__ float ldv(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// floor(p) = P >> F; the FP32 path has F = 32, so it is the high word.
template <typename T>
__device__ __forceinline__ int bin_of(long long P, int F)
{
    if constexpr (sizeof(T) == 4) return (int)(P >> 32);
    else return (int)(P >> F);
}

#ifndef CTR_FWD_UNROLL
#define CTR_FWD_UNROLL 8
#endif
constexpr int FWD_UNROLL = CTR_FWD_UNROLL;   // rows per unrolled step of the ray march
#ifndef CTR_FWD_UNROLL_ORBIT
#define CTR_FWD_UNROLL_ORBIT 8
#endif
constexpr int FWD_UNROLL_ORBIT = CTR_FWD_UNROLL_ORBIT;

// x / d for x, d >= 0 with x d < 2^32 as the high word of x m, m = floor((2^32 - 1) / d) + 1
// (then m - 2^32 / d < 1 and the error x (m - 2^32/d) / 2^32 stays below 1/d, so the floor is
// exact).  The staging loops divide element indices by a row width once per copied element;
// a runtime integer division costs an instruction sequence, this one multiply.
__device__ __forceinline__ unsigned udiv_magic(unsigned d) { return d <= 1 ? 0u : 0xFFFFFFFFu / d + 1u; }
__device__ __forceinline__ int udiv_fast(int x, int d, unsigned m) { return d <= 1 ? x : (int)__umulhi((unsigned)x, m); }

// 1 + frac(p) in [1, 2) from the low 32 bits of P (F = 32): the top 23 fraction
// bits become the mantissa of a float, so the weight is exact and identical in
// both projectors.
__device__ __forceinline__ float one_plus_frac32(long long P)
{
    return __uint_as_float((((unsigned)(unsigned long long)P) >> 9) | 0x3F800000u);
}

__device__ __forceinline__ float one_plus_frac32u(unsigned lo)
{
    return __uint_as_float((lo >> 9) | 0x3F800000u);
}

__device__ __forceinline__ float2 make_stage(float g0, float g1)
{
    const float d = g1 - g0;
    return make_float2(g0 - d, d);     // value = (g0 - d) + (1 + frac) d
}
__device__ __forceinline__ double2 make_stage(double g0, double g1)
{
    return make_double2(g0, g1 - g0);  // value = g0 + frac d
}

__device__ __forceinline__ float interp(float acc, float2 pr, long long P, int, double)
{
    return fmaf(one_plus_frac32(P), pr.y, acc + pr.x);
}
__device__ __forceinline__ double interp(double acc, double2 pr, long long P, int F, double inv2F)
{
    const unsigned long long mask = (1ull << F) - 1ull;
    const double a = (double)((unsigned long long)P & mask) * inv2F;
    return acc + fma(a, pr.y, pr.x);
}

template <typename T>
__device__ __forceinline__ void bp_epilogue(const BackprojEpi<T> &epi, int n, int i, int j, T acc)
{
    const size_t o = (size_t)i * n + j;
    const T old = epi.bar_out ? epi.ub[o] : T(0);      // read before out (may alias ub) is written
    const T v = bp_epilogue_value(epi, n, i, j, acc);
    if (epi.bar_out) epi.bar_out[o] = T(2) * v - old;
    if (epi.complex_out) {
        epi.out[2 * o] = v;
        epi.out[2 * o + 1] = T(0);
    } else {
        epi.out[o] = v;
    }
}

// One CTA of the backprojection: tile (bx, by), angle group bz.
// part == nullptr: apply the epilogue directly (one angle group).  Otherwise write
// this group's partial sums to part[bz][n][n].
template <typename T, typename S, bool NAMED = false>
__device__ __forceinline__ void bp_body(const S *__restrict__ g, int n, int N, int M, int F, int wstride,
                                        int angles_per_group, const AngleGeom *__restrict__ geom,
                                        const BackprojEpi<T> &epi, T *__restrict__ part, int bx, int by, int bz)
{
    using T2 = typename Pair<T>::type;
    constexpr int NT = 32 * BP_TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *stage = reinterpret_cast<T2 *>(smem_raw);
    long long *sPb = reinterpret_cast<long long *>(stage + BP_ACH * wstride);
    long long *sC = sPb + BP_ACH;
    long long *sS = sC + BP_ACH;
    int *sK = reinterpret_cast<int *>(sS + BP_ACH);

    const int tx = threadIdx.x & 31;
    const int ty = threadIdx.x >> 5;
    const int i0 = by * BP_TI;
    const int j0 = bx * BP_TJ;
    const int la = bz * angles_per_group;
    const int lb = min(N, la + angles_per_group);
    const double inv2F = ldexp(1.0, -F);

    T acc[BP_R];
#pragma unroll
    for (int r = 0; r < BP_R; ++r) acc[r] = T(0);

    for (int l0 = la; l0 < lb; l0 += BP_ACH) {
        const int na = min(BP_ACH, lb - l0);
        body_sync<NAMED>();
        if (threadIdx.x < na) {
            const AngleGeom ag = geom[l0 + threadIdx.x];
            const long long P00 = (long long)i0 * ag.C + (long long)j0 * ag.S + ag.O;
            const long long P10 = P00 + (long long)(BP_TI - 1) * ag.C;
            const long long P01 = P00 + (long long)(BP_TJ - 1) * ag.S;
            const long long P11 = P10 + (long long)(BP_TJ - 1) * ag.S;
            const long long pmin = min(min(P00, P10), min(P01, P11));
            const long long kmin = pmin >> F;   // arithmetic shift: floor
            sK[threadIdx.x] = (int)kmin;
            sPb[threadIdx.x] = P00 - (kmin << F);
            sC[threadIdx.x] = ag.C;
            sS[threadIdx.x] = ag.S;
        }
        body_sync<NAMED>();
        const unsigned mw = udiv_magic((unsigned)wstride);
        for (int e = threadIdx.x; e < na * wstride; e += NT) {
            const int a = udiv_fast(e, wstride, mw);
            const int k = sK[a] + (e - a * wstride);
            const S *row = g + (size_t)(l0 + a) * M;
            const T g0 = (k >= 0 && k < M) ? (T)ldv(row + k) : T(0);
            const T g1 = (k + 1 >= 0 && k + 1 < M) ? (T)ldv(row + k + 1) : T(0);
            stage[e] = make_stage(g0, g1);
        }
        body_sync<NAMED>();
#pragma unroll 2
        for (int a = 0; a < na; ++a) {
            const long long C = sC[a];
            long long P = sPb[a] + (long long)ty * C + (long long)tx * sS[a];
            const long long D = C * BP_TY;
            const T2 *row = stage + a * wstride;
#pragma unroll
            for (int r = 0; r < BP_R; ++r) {
                acc[r] = interp(acc[r], row[bin_of<T>(P, F)], P, F, inv2F);
                P += D;
            }
        }
    }

    const int j = j0 + tx;
#pragma unroll
    for (int r = 0; r < BP_R; ++r) {
        const int i = i0 + ty + BP_TY * r;
        if (i < n && j < n) {
            if (part) part[((size_t)bz * n + i) * n + j] = acc[r];
            else bp_epilogue(epi, n, i, j, acc[r]);
        }
    }
}

template <typename T, typename S>
__global__ void __launch_bounds__(32 * BP_TY)
k_backproject(const S *__restrict__ g, int n, int N, int M, int F, int wstride, int angles_per_group,
              const AngleGeom *__restrict__ geom, BackprojEpi<T> epi, T *__restrict__ part)
{
    bp_body<T, S>(g, n, N, M, F, wstride, angles_per_group, geom, epi, part, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Sum of the angle groups' partial images, then the backprojection epilogue
// (block b of nb, grid-stride over the n*n pixels).
template <typename T>
__device__ __forceinline__ void bp_reduce_body(const T *__restrict__ part, int groups, int n,
                                               const BackprojEpi<T> &epi, int b, int nb)
{
    const size_t nn = (size_t)n * n;
    for (size_t e = b * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)nb * blockDim.x) {
        T s = part[e];
        for (int z = 1; z < groups; ++z) s += part[(size_t)z * nn + e];
        bp_epilogue(epi, n, pix_i(e, n), pix_j(e, n), s);
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_bp_reduce(const T *__restrict__ part, int groups, int n, BackprojEpi<T> epi)
{
    bp_reduce_body<T>(part, groups, n, epi, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ long long ceil_div_ll(long long a, long long b)
{
    // b > 0
    long long q = a / b;
    if (q * b < a) ++q;
    return q;
}

__device__ __forceinline__ void acc_sample(float &Su, float &Sf, float v, long long P, int, double)
{
    Su += v;
    Sf = fmaf(one_plus_frac32(P), v, Sf);     // sum (1 + frac) u
}
__device__ __forceinline__ void acc_sample(double &Su, double &Sf, double v, long long P, int F, double inv2F)
{
    const unsigned long long mask = (1ull << F) - 1ull;
    Su += v;
    Sf = fma((double)((unsigned long long)P & mask) * inv2F, v, Sf);   // sum frac u
}

// The data resolvent (id + s dg_r^*)^{-1}(z) = z - s clip(q, lo, hi), q = (z + w a)/(s + w),
// written as w (z - s a)/(s + w) + s (q - clip(q)): for w = 0 and q inside the box it is
// exactly 0 (the one-sided trace constraint then keeps its dual in the conjugate's domain).
template <typename T>
__device__ __forceinline__ T data_resolvent(T z, T s, T w, T a, T lo, T hi)
{
    const T q = (z + w * a) / (s + w);
    return w * (z - s * a) / (s + w) + s * (q - fmin(fmax(q, lo), hi));
}

template <typename T>
__device__ __forceinline__ void forward_epilogue(const ForwardEpi<T> &epi, size_t r, T val)
{
    if (epi.mode == 0) {
        epi.g[r] = val * epi.scale;
        return;
    }
    if (epi.mode == 2) {
        // Alg. 1: v = (id + tau dG1^*)^{-1}(v + tau Rt u_bar), tau carried in epi.sigma
        const T z = epi.v1b[r] + epi.sigma * (val * epi.scale);
        epi.v1b[r] = data_resolvent(z, epi.sigma, epi.dw[r], epi.da[r], epi.dlo[r], epi.dhi[r]);
        return;
    }
    if (epi.mode == 3) {
        // Alg. 3: the next iteration backprojects the residual Rt u_new - ft
        const T Ru = val * epi.scale;
        const T y = Ru - epi.da[r];
        epi.Ru[r] = Ru;
        if constexpr (sizeof(T) == 4) {
            if (epi.y1h) epi.y1h[r] = __float2bfloat16_rn(y);
            else epi.y1[r] = y;
        } else {
            epi.y1[r] = y;
        }
        if (epi.t1) epi.t1[r] = y;
        return;
    }
    // Alg. 4: v1 = v1b + sigma Rt u_new; t = (id + sigma dG1^*)^{-1}(2 v1 - v1b);
    // v1b <- v1b + t - v1; and the next iteration's y1 = v1b + sigma Rt u_new.
    const T sigma = epi.sigma;
    const T Ru = val * epi.scale;
    const T vb = epi.v1b[r];
    const T v1 = vb + sigma * Ru;
    const T z = T(2) * v1 - vb;
    const T t = data_resolvent(z, sigma, epi.dw[r], epi.da[r], epi.dlo[r], epi.dhi[r]);
    const T vbn = vb + t - v1;
    epi.Ru[r] = Ru;
    epi.v1b[r] = vbn;
    if constexpr (sizeof(T) == 4) {
        if (epi.y1h) epi.y1h[r] = __float2bfloat16_rn(vbn + sigma * Ru);
        else epi.y1[r] = vbn + sigma * Ru;
    } else {
        epi.y1[r] = vbn + sigma * Ru;
    }
    if (epi.t1) epi.t1[r] = t;
}

// The same epilogue (modes 1 and 2) on operands fetched ahead: vb = v1b[r], w, a, lo, hi.
__device__ __forceinline__ void forward_epilogue_pre(const ForwardEpi<float> &epi, size_t r, float val, float vb,
                                                     float w, float a, float lo, float hi)
{
    const float sigma = epi.sigma;
    if (epi.mode == 2) {
        const float z = vb + sigma * (val * epi.scale);
        epi.v1b[r] = data_resolvent(z, sigma, w, a, lo, hi);
        return;
    }
    const float Ru = val * epi.scale;
    const float v1 = vb + sigma * Ru;
    const float z = 2.f * v1 - vb;
    const float t = data_resolvent(z, sigma, w, a, lo, hi);
    const float vbn = vb + t - v1;
    epi.Ru[r] = Ru;
    epi.v1b[r] = vbn;
    if (epi.y1h) epi.y1h[r] = __float2bfloat16_rn(vbn + sigma * Ru);
    else epi.y1[r] = vbn + sigma * Ru;
    if (epi.t1) epi.t1[r] = t;
}

// One row of the march: the NC candidate pixels q, q+1, ... of the lane's interval.
// EXACT1: the first candidate is always inside the interval (A <= 2^F, i.e. h <= ds).
template <typename T, typename S, int NC, bool EXACT1>
__device__ __forceinline__ void march_row(const S *__restrict__ rowp, int dq, int n, int k, int F, double inv2F,
                                          long long Pa, int q, long long A, T &Su, T &Sf)
{
    {
        bool ok = (unsigned)q < (unsigned)n;
        if (!EXACT1) ok = ok && bin_of<T>(Pa, F) == k;
        const T v = ok ? (T)ldv(rowp + dq * q) : T(0);
        acc_sample(Su, Sf, v, Pa, F, inv2F);
    }
    long long P = Pa;
#pragma unroll
    for (int c = 1; c < NC; ++c) {
        P += A;
        const int qq = q + c;
        const bool ok = bin_of<T>(P, F) == k && (unsigned)qq < (unsigned)n;
        if (__any_sync(0xffffffffu, ok)) {
            const T v = ok ? (T)ldv(rowp + dq * qq) : T(0);
            acc_sample(Su, Sf, v, P, F, inv2F);
        }
    }
}

constexpr int FWD_AW = 4;                     // adjacent angles per CTA, one warp each
constexpr int FWD_THREADS = 32 * FWD_AW;

// FP32 ray march over `rows` rows (F = 32, 2^31 <= A <= 2^32).  State: r = P(q_a) - k 2^32
// in [0, A) (the fixed-point fraction of the interval's first pixel q_a), off = element
// offset of pixel (m, q_a), and q_a itself where CHECK.  The second pixel q_a + 1 lies in
// the interval iff r + A < 2^32, i.e. r < lim.  Next row: P += B; B > 0 (BPOS) steps
// q_a back when r >= thr = A - B, B <= 0 steps it forward when r < thr = |B|.
// CHECK = false: every lane's q_a and q_a + 1 are inside [0, n) on these rows.
template <int DQ, bool BPOS, bool CHECK, typename S>
__device__ __forceinline__ void march32(const S *__restrict__ base, int n, int rows, unsigned &r, int &q, int &off,
                                        unsigned A32, unsigned lim, unsigned B32, unsigned thr, float &Su, float &Sf)
{
#pragma unroll FWD_UNROLL
    for (int rr = 0; rr < rows; ++rr) {
        float v1, v2;
        if constexpr (CHECK) {
            v1 = ((unsigned)q < (unsigned)n) ? ldv(base + off) : 0.f;
            v2 = (r < lim && (unsigned)(q + 1) < (unsigned)n) ? ldv(base + off + DQ) : 0.f;
        } else {
            v1 = ldv(base + off);
            v2 = r < lim ? ldv(base + off + DQ) : 0.f;
        }
        Su += v1 + v2;
        Sf = fmaf(one_plus_frac32u(r), v1, Sf);
        Sf = fmaf(one_plus_frac32u(r + A32), v2, Sf);
        if constexpr (BPOS) {
            const bool s = r >= thr;
            r += s ? B32 - A32 : B32;
            off += s ? n - DQ : n;
            if constexpr (CHECK) q -= s ? 1 : 0;
        } else {
            const bool s = r < thr;
            r += s ? A32 - thr : 0u - thr;
            off += s ? n + DQ : n;
            if constexpr (CHECK) q += s ? 1 : 0;
        }
    }
}

// The FP32 march of one lane over rows [mlo, mhi] of the warp, without bounds checks on
// the warp's interior rows [ilo, ihi] (mlo <= ilo, ihi <= mhi; ilo > ihi: none).
template <int DQ, bool BPOS, typename S>
__device__ __forceinline__ void march32_rows(const S *__restrict__ base, int n, long long K, const AngleMarch &am,
                                             int mlo, int mhi, int ilo, int ihi, float &Su, float &Sf)
{
    const long long A = am.A, B = am.B;
    const long long qa = ceil_div_ll(K - (long long)mlo * B - am.Op, A);
    unsigned r = (unsigned)(qa * A + (long long)mlo * B + am.Op - K);
    int q = (int)qa;
    int off = mlo * n + DQ * q;
    const unsigned A32 = (unsigned)A;             // A = 2^32 wraps to 0 (then B = 0)
    const unsigned lim = (unsigned)((1ll << 32) - A);
    const unsigned B32 = (unsigned)B;
    const unsigned thr = BPOS ? (unsigned)(A - B) : (unsigned)(-B);
    if (ilo > ihi) {
        march32<DQ, BPOS, true>(base, n, mhi - mlo + 1, r, q, off, A32, lim, B32, thr, Su, Sf);
        return;
    }
    march32<DQ, BPOS, true>(base, n, ilo - mlo, r, q, off, A32, lim, B32, thr, Su, Sf);
    march32<DQ, BPOS, false>(base, n, ihi - ilo + 1, r, q, off, A32, lim, B32, thr, Su, Sf);
    q = DQ * (off - (ihi + 1) * n);               // off = m n + DQ q
    march32<DQ, BPOS, true>(base, n, mhi - ihi, r, q, off, A32, lim, B32, thr, Su, Sf);
}

// Sum u and sum frac u (FP64) or sum (1 + frac) u (generic FP32) over the pixels of rows
// m0 .. m0 + rows - 1 whose detector coordinate lies in the lane's interval [k, k+1).
template <typename T, typename S, int NC, bool EXACT1>
__device__ __forceinline__ void fwd_march(const S *__restrict__ base, int dq, int n, int k, int F,
                                          const AngleMarch &am, int m0, int rows, T &Su, T &Sf)
{
    const double inv2F = ldexp(1.0, -F);
    const long long K = (long long)k << F;
    const long long A = am.A, B = am.B;
    long long qa = ceil_div_ll(K - (long long)m0 * B - am.Op, A);
    long long Pa = qa * A + (long long)m0 * B + am.Op;   // in [K, K + A)
    int q = (int)qa;
    const S *rowp = base + (size_t)m0 * n;
    // next row: restore P(q_a) in [K, K + A) (|B| <= A: at most one step)
    if (B >= 0) {
        const long long KA = K + A;
#pragma unroll 2
        for (int r = 0; r < rows; ++r) {
            march_row<T, S, NC, EXACT1>(rowp, dq, n, k, F, inv2F, Pa, q, A, Su, Sf);
            Pa += B;
            if (Pa >= KA) { Pa -= A; --q; }
            rowp += n;
        }
    } else {
#pragma unroll 2
        for (int r = 0; r < rows; ++r) {
            march_row<T, S, NC, EXACT1>(rowp, dq, n, k, F, inv2F, Pa, q, A, Su, Sf);
            Pa += B;
            if (Pa < K) { Pa += A; ++q; }
            rowp += n;
        }
    }
}

// Rows m of [0, n) on which q*(m) = Q0 - m b lies in [qlo, qhi] (FP32; the callers'
// margins of half a pixel or more absorb its rounding).  OUTER rounds the range out
// (rows that may touch), otherwise in (rows that surely lie inside).  lo > hi: none.
template <bool OUTER>
__device__ __forceinline__ void rows_in(float Q0, float binv, float qlo, float qhi, int n, int &lo, int &hi)
{
    lo = n;
    hi = -1;
    if (qlo > qhi) return;
    if (binv != 0.f) {
        const float m1 = (Q0 - qhi) * binv, m2 = (Q0 - qlo) * binv;
        float a0 = fminf(m1, m2), a1 = fmaxf(m1, m2);
        a0 = fmaxf(0.f, OUTER ? floorf(a0) : ceilf(a0));
        a1 = fminf((float)(n - 1), OUTER ? ceilf(a1) : floorf(a1));
        if (a0 <= a1) {
            lo = (int)a0;
            hi = (int)a1;
        }
    } else if (Q0 > qlo && Q0 < qhi) {            // rays parallel to the march axis
        lo = 0;
        hi = n - 1;
    }
}

// One CTA of the forward projector: warp w takes angle by*FWD_AW + w and bins
// bx*31 + [0, 31).  The angles are adjacent, so their rays nearly coincide and the
// image rows they read are shared in L1.
template <typename T, typename S, int NC, bool EXACT1>
__device__ __forceinline__ void fwd_body(const S *__restrict__ u, const S *__restrict__ uT, int n, int N, int M, int F,
                                         const AngleMarch *__restrict__ march, const ForwardEpi<T> &epi, int bx, int by)
{
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int l = by * FWD_AW + warp;
    const int kb = bx * 31;                           // first output bin of this warp
    const int k = kb + lane - 1;                      // this lane's interval [k, k+1)
    if (l >= N || kb >= M) return;                    // warp-uniform
    const AngleMarch am = march[l];
    // pixel (m, q) of the march is at base[m*n + dq*q]
    const S *__restrict__ base = (am.layout ? u : uT) + (am.flip ? (n - 1) : 0);
    // q*(m) = Q0 - m b: the real pick coordinate where P(q, m) = k 2^F
    const float Q0 = (float)k * am.kA - am.oA;
    int mlo, mhi;                                     // rows where the lane's pixel run may be inside [0, n)
    rows_in<true>(Q0, am.binv, -(float)NC - 1.f, (float)n + 1.f, n, mlo, mhi);
    const int mlo_w = __reduce_min_sync(0xffffffffu, mlo);
    const int mhi_w = __reduce_max_sync(0xffffffffu, mhi);
    T Su = T(0), Sf = T(0);
    if (mlo_w <= mhi_w) {
        if constexpr (sizeof(T) == 4 && EXACT1 && NC == 2) {
            // interior rows: q_a in [1, n - 3] for every lane, no bounds checks needed
            int ilo, ihi;
            rows_in<false>(Q0, am.binv, 0.5f, (float)n - 3.5f, n, ilo, ihi);
            const int ilo_w = max(__reduce_max_sync(0xffffffffu, ilo), mlo_w);
            const int ihi_w = min(__reduce_min_sync(0xffffffffu, ihi), mhi_w);
            const long long K = (long long)k << 32;
            if (am.B > 0) {                           // B = 0 takes the B < 0 march (thr = 0: never steps)
                if (am.flip) march32_rows<-1, true>(base, n, K, am, mlo_w, mhi_w, ilo_w, ihi_w, Su, Sf);
                else march32_rows<1, true>(base, n, K, am, mlo_w, mhi_w, ilo_w, ihi_w, Su, Sf);
            } else {
                if (am.flip) march32_rows<-1, false>(base, n, K, am, mlo_w, mhi_w, ilo_w, ihi_w, Su, Sf);
                else march32_rows<1, false>(base, n, K, am, mlo_w, mhi_w, ilo_w, ihi_w, Su, Sf);
            }
        } else {
            fwd_march<T, S, NC, EXACT1>(base, am.flip ? -1 : 1, n, k, F, am, mlo_w, mhi_w - mlo_w + 1, Su, Sf);
        }
    }
    T Bk, Ak;
    if constexpr (sizeof(T) == 4) { Bk = Sf - Su; Ak = Su - Bk; }
    else { Bk = Sf; Ak = Su - Sf; }
    const T Bprev = __shfl_up_sync(0xffffffffu, Bk, 1);
    if (lane >= 1 && k < M) forward_epilogue(epi, (size_t)l * M + k, Ak + Bprev);
}

template <typename T, typename S, int NC, bool EXACT1>
__global__ void __launch_bounds__(FWD_THREADS)
k_forward(const S *__restrict__ u, const S *__restrict__ uT, int n, int N, int M, int F,
          const AngleMarch *__restrict__ march, ForwardEpi<T> epi)
{
    fwd_body<T, S, NC, EXACT1>(u, uT, n, N, M, F, march, epi, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Symmetric forward path (OrbitJob): one canonical ray march per job serves the
// job's up to four angles, reading the four channels of the orbit image at once.
// ---------------------------------------------------------------------------

// Orbit-image records: the four channels of one pixel, FP32 (float4) or bfloat16
// (uint2, channel 0 in the low half of x).  rec_f32 widens a record to FP32.
template <typename S> struct OrbitRec;
template <> struct OrbitRec<float> { using type = float4; };
template <> struct OrbitRec<__nv_bfloat16> { using type = uint2; };
__device__ __forceinline__ float4 rec_f32(float4 v) { return v; }
__device__ __forceinline__ float4 rec_f32(uint2 v)
{
    return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xFFFF0000u), __uint_as_float(v.y << 16),
                       __uint_as_float(v.y & 0xFFFF0000u));
}
__device__ __forceinline__ float4 make_rec(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
__device__ __forceinline__ uint2 make_rec(__nv_bfloat16 a, __nv_bfloat16 b, __nv_bfloat16 c, __nv_bfloat16 d)
{
    return make_uint2((unsigned)__bfloat16_as_ushort(a) | ((unsigned)__bfloat16_as_ushort(b) << 16),
                      (unsigned)__bfloat16_as_ushort(c) | ((unsigned)__bfloat16_as_ushort(d) << 16));
}

// ubar[m][q] = (u[q][m], u[n-1-q][m], u[m][q], u[n-1-m][q]): channel v holds
// u(T_v^{-1}(q, m)) for the canonical march pixel (q, m) (pick q = i, march m = j).
// 32 x 32 tiles: four coalesced tile loads (two of them transposed through shared
// memory), one coalesced record store per pixel.
template <typename S>
__device__ __forceinline__ void orbit_image_body(const S *__restrict__ u, typename OrbitRec<S>::type *__restrict__ ubar,
                                                 int n, int bx, int by)
{
    __shared__ S tA[32][33], tB[32][33], tC[32][33], tD[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int q0 = bx * 32, m0 = by * 32;
    for (int r = ty; r < 32; r += 8) {
        const int mr = m0 + r, qc = q0 + tx;          // tiles A, B: rows m, columns q
        if (mr < n && qc < n) {
            tA[r][tx] = u[(size_t)mr * n + qc];
            tB[r][tx] = u[(size_t)(n - 1 - mr) * n + qc];
        }
        const int qr = q0 + r, mc = m0 + tx;          // tiles C, D: rows q, columns m
        if (qr < n && mc < n) {
            tC[r][tx] = u[(size_t)qr * n + mc];
            tD[r][tx] = u[(size_t)(n - 1 - qr) * n + mc];
        }
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int m = m0 + r, q = q0 + tx;
        if (m < n && q < n) ubar[(size_t)m * n + q] = make_rec(tC[tx][r], tD[tx][r], tA[r][tx], tB[r][tx]);
    }
}

template <typename S>
__global__ void __launch_bounds__(256)
k_orbit_image(const S *__restrict__ u, typename OrbitRec<S>::type *__restrict__ ubar, int n)
{
    pdl_wait();
    pdl_trigger();
    orbit_image_body<S>(u, ubar, n, blockIdx.x, blockIdx.y);
}

// The orbit image and, for the pixels (m, q) of the CTA's tile, the TV dual step of
// Alg. 4 (both read u; each pixel's TV step runs exactly once over the grid).  The TV
// operands (bar v2, and bar u for Alg. 5) are fetched before the tile barrier, and u with
// its forward neighbours comes from tile A (rows m, columns q, plus a one-pixel halo), so
// the kernel waits on global memory once; the arithmetic is that of tv_dual_at.
__global__ void __launch_bounds__(256)
k_orbit_image_tv(const float *__restrict__ u, OrbitRec<float>::type *__restrict__ ubar, int n, TvDualJob<float> tv)
{
    pdl_wait();
    pdl_trigger();
    __shared__ float tA[33][33], tB[32][33], tC[32][33], tD[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int q0 = blockIdx.x * 32, m0 = blockIdx.y * 32;
    const size_t nn = (size_t)n * n;
    float vbx[4], vby[4], ubv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int m = m0 + ty + 8 * k, q = q0 + tx;
        vbx[k] = vby[k] = ubv[k] = 0.f;
        if (m < n && q < n) {
            const size_t e = (size_t)m * n + q;
            vbx[k] = tv.v2b[e];
            vby[k] = tv.v2b[e + nn];
            if (tv.ub) ubv[k] = tv.ub[e];
        }
    }
    for (int r = ty; r < 32; r += 8) {
        const int mr = m0 + r, qc = q0 + tx;          // tiles A, B: rows m, columns q
        if (mr < n && qc < n) {
            tA[r][tx] = u[(size_t)mr * n + qc];
            tB[r][tx] = u[(size_t)(n - 1 - mr) * n + qc];
        }
        const int qr = q0 + r, mc = m0 + tx;          // tiles C, D: rows q, columns m
        if (qr < n && mc < n) {
            tC[r][tx] = u[(size_t)qr * n + mc];
            tD[r][tx] = u[(size_t)(n - 1 - qr) * n + mc];
        }
    }
    if (ty == 0 && m0 + 32 < n && q0 + tx < n) tA[32][tx] = u[(size_t)(m0 + 32) * n + q0 + tx];   // halo row
    if (ty == 1 && q0 + 32 < n && m0 + tx < n) tA[tx][32] = u[(size_t)(m0 + tx) * n + q0 + 32];   // halo column
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int m = m0 + r, q = q0 + tx;
        if (m < n && q < n) ubar[(size_t)m * n + q] = make_rec(tC[tx][r], tD[tx][r], tA[r][tx], tB[r][tx]);
    }
    const float st = tv.sigma * tv.tau;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = ty + 8 * k, m = m0 + r, q = q0 + tx;
        if (m >= n || q >= n) continue;
        const size_t e = (size_t)m * n + q;
        const float c = tA[r][tx];
        const float gx = (m < n - 1) ? (tA[r + 1][tx] - c) * tv.inv_h : 0.f;
        const float gy = (q < n - 1) ? (tA[r][tx + 1] - c) * tv.inv_h : 0.f;
        const float bx = vbx[k], by = vby[k];
        const float vx = bx + st * gx, vy = by + st * gy;
        const float zx = 2.f * vx - bx, zy = 2.f * vy - by;
        float tx2 = 0.f, ty2 = 0.f;
        if (tv.lam > 0.f) {
            const float den = fmax(1.f, tv.tau * sqrt(zx * zx + zy * zy) / tv.lam);
            tx2 = zx / den;
            ty2 = zy / den;
        }
        const float nbx = bx + tx2 - vx, nby = by + ty2 - vy;
        tv.v2b[e] = nbx;
        tv.v2b[e + nn] = nby;
        tv.y2[e] = nbx + st * gx;
        tv.y2[e + nn] = nby + st * gy;
        if (tv.t2) {
            tv.t2[e] = tx2;
            tv.t2[e + nn] = ty2;
        }
        if (tv.ub) tv.ub[e] = ubv[k] + fmax(2.f * c - ubv[k], 0.f) - c;
    }
}

// Asynchronous copies global -> shared (cp.async): one 4-byte element (src_size 0 stores
// zero and reads nothing), commit and wait on this thread's groups.
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Paired FP32 arithmetic (add / sub / fma on two lanes of a 64-bit register pair, one
// instruction for two values; each lane rounds exactly as the scalar instruction).
#ifndef CTR_F32X2
#define CTR_F32X2 1
#endif
__device__ __forceinline__ float2 fadd2(float2 a, float2 b)
{
#if CTR_F32X2
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__device__ __forceinline__ float2 fsub2(float2 a, float2 b)
{
#if CTR_F32X2
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
#else
    return make_float2(a.x - b.x, a.y - b.y);
#endif
}
// a * b + c per lane
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c)
{
#if CTR_F32X2
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
#else
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}

__device__ __forceinline__ void acc4(float4 &Su, float4 &Sf, float4 v, float f)
{
#if CTR_F32X2
    const float2 f2 = make_float2(f, f);
    const float2 v01 = make_float2(v.x, v.y), v23 = make_float2(v.z, v.w);
    const float2 u01 = fadd2(make_float2(Su.x, Su.y), v01), u23 = fadd2(make_float2(Su.z, Su.w), v23);
    const float2 s01 = ffma2(f2, v01, make_float2(Sf.x, Sf.y)), s23 = ffma2(f2, v23, make_float2(Sf.z, Sf.w));
    Su = make_float4(u01.x, u01.y, u23.x, u23.y);
    Sf = make_float4(s01.x, s01.y, s23.x, s23.y);
    return;
#endif
    Su.x += v.x;
    Su.y += v.y;
    Su.z += v.z;
    Su.w += v.w;
    Sf.x = fmaf(f, v.x, Sf.x);
    Sf.y = fmaf(f, v.y, Sf.y);
    Sf.z = fmaf(f, v.z, Sf.z);
    Sf.w = fmaf(f, v.w, Sf.w);
}

// What the march reads at a pixel: the whole orbit record (four channels), or for a pair
// job (whose angles all sit in channels {0, 1} or {2, 3}) the two live channels of the
// FP32 record as one 8-byte load.  acc_v accumulates each channel exactly as acc4 does.
template <typename R>
struct RecLoad {
    using V = float4;
    const R *__restrict__ ub;
    __device__ __forceinline__ float4 operator()(int off) const { return rec_f32(ub[off]); }
    __device__ __forceinline__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
struct PairLoad {
    using V = float2;
    const float2 *__restrict__ ub2;     // (const float2 *)ub + h: channels 2h, 2h + 1 of each record
    __device__ __forceinline__ float2 operator()(int off) const { return ub2[2 * (size_t)off]; }
    __device__ __forceinline__ static float2 zero() { return make_float2(0.f, 0.f); }
};
__device__ __forceinline__ void acc_v(float4 &Su, float4 &Sf, float4 v, float f) { acc4(Su, Sf, v, f); }
__device__ __forceinline__ void acc_v(float2 &Su, float2 &Sf, float2 v, float f)
{
    Su = fadd2(Su, v);
    Sf = ffma2(make_float2(f, f), v, Sf);
}

// The canonical march (flip 0, B >= 0) over `rows` rows of the orbit image; the
// state and the second-pixel rule are those of march32.
template <bool BPOS, bool CHECK, typename L>
__device__ __forceinline__ void march_orbit(const L &ld, int n, int rows, unsigned &r, int &q, int &off,
                                            unsigned A32, unsigned lim, unsigned B32, unsigned thr,
                                            typename L::V &Su, typename L::V &Sf)
{
    using V = typename L::V;
#pragma unroll FWD_UNROLL_ORBIT
    for (int rr = 0; rr < rows; ++rr) {
        V v1, v2;
        if constexpr (CHECK) {
            v1 = ((unsigned)q < (unsigned)n) ? ld(off) : L::zero();
            v2 = (r < lim && (unsigned)(q + 1) < (unsigned)n) ? ld(off + 1) : L::zero();
        } else {
            v1 = ld(off);
            v2 = r < lim ? ld(off + 1) : L::zero();
        }
        acc_v(Su, Sf, v1, one_plus_frac32u(r));
        acc_v(Su, Sf, v2, one_plus_frac32u(r + A32));
        if constexpr (BPOS) {
            const bool s = r >= thr;
            r += s ? B32 - A32 : B32;
            off += s ? n - 1 : n;
            if constexpr (CHECK) q -= s ? 1 : 0;
        } else {
            const bool s = r < thr;
            r += s ? A32 - thr : 0u - thr;
            off += s ? n + 1 : n;
            if constexpr (CHECK) q += s ? 1 : 0;
        }
    }
}

template <bool BPOS, typename L>
__device__ __forceinline__ void march_orbit_rows(const L &ub, int n, long long K, const AngleMarch &am, int mlo,
                                                 int mhi, int ilo, int ihi, typename L::V &Su, typename L::V &Sf)
{
    const long long A = am.A, B = am.B;
    const long long qa = ceil_div_ll(K - (long long)mlo * B - am.Op, A);
    unsigned r = (unsigned)(qa * A + (long long)mlo * B + am.Op - K);
    int q = (int)qa;
    int off = mlo * n + q;
    const unsigned A32 = (unsigned)A;
    const unsigned lim = (unsigned)((1ll << 32) - A);
    const unsigned B32 = (unsigned)B;
    const unsigned thr = BPOS ? (unsigned)(A - B) : (unsigned)(-B);
    if (ilo > ihi) {
        march_orbit<BPOS, true>(ub, n, mhi - mlo + 1, r, q, off, A32, lim, B32, thr, Su, Sf);
        return;
    }
    march_orbit<BPOS, true>(ub, n, ilo - mlo, r, q, off, A32, lim, B32, thr, Su, Sf);
    march_orbit<BPOS, false>(ub, n, ihi - ilo + 1, r, q, off, A32, lim, B32, thr, Su, Sf);
    q = off - (ihi + 1) * n;
    march_orbit<BPOS, true>(ub, n, mhi - ihi, r, q, off, A32, lim, B32, thr, Su, Sf);
}

__device__ __forceinline__ void orbit_out(const ForwardEpi<float> &epi, int l, int M, int k, int lane, float Su,
                                          float Sf, const float *pre = nullptr)
{
    const float Bk = Sf - Su, Ak = Su - Bk;
    const float Bprev = __shfl_up_sync(0xffffffffu, Bk, 1);
    if (l >= 0 && lane >= 1 && k < M) {
        if (pre) forward_epilogue_pre(epi, (size_t)l * M + k, Ak + Bprev, pre[0], pre[32], pre[64], pre[96], pre[128]);
        else forward_epilogue(epi, (size_t)l * M + k, Ak + Bprev);
    }
}

// The data-dual epilogue's per-bin operands (v1b, w, a, lo, hi) of the lane's four angles,
// copied into shared memory [angle][operand][lane] at the start of the march so that their
// latency is hidden behind it (modes 1 and 2 read them; each (angle, bin) belongs to one lane).
__device__ __forceinline__ void orbit_epi_prefetch(const ForwardEpi<float> &epi, int4 ls, int M, int k, int lane,
                                                   float *s)
{
    const int l4[4] = {ls.x, ls.y, ls.z, ls.w};
    const float *src[5] = {epi.v1b, epi.dw, epi.da, epi.dlo, epi.dhi};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const bool ok = l4[c] >= 0 && lane >= 1 && k < M;
        const size_t r = ok ? (size_t)l4[c] * M + k : 0;
#pragma unroll
        for (int o = 0; o < 5; ++o) cp_async4(s + (c * 5 + o) * 32 + lane, src[o] + r, ok);
    }
    cp_async_commit();
}

#ifndef CTR_ORBIT_SEGS
#define CTR_ORBIT_SEGS 4
#endif
constexpr int ORBIT_SEGS = CTR_ORBIT_SEGS;    // row segments of a job's rays (one warp each)
#ifndef CTR_ORBIT_SLOTS
#define CTR_ORBIT_SLOTS 1
#endif
// adjacent jobs per CTA; 1 (128-thread CTAs, 8 per SM) measured fastest: co-resident CTAs of
// adjacent jobs share the SM's L1 anyway, and small CTAs retire and refill sooner
constexpr int ORBIT_SLOTS = CTR_ORBIT_SLOTS;
constexpr int ORBIT_THREADS = 32 * ORBIT_SLOTS * ORBIT_SEGS;
#ifndef CTR_ORBIT_MINB
#define CTR_ORBIT_MINB 8
#endif
#ifndef CTR_OBP_MINB
#define CTR_OBP_MINB 4
#endif

// Warp w of the CTA takes job by*ORBIT_SLOTS + w % ORBIT_SLOTS, bins bx*31 + [0, 31) and
// the (w / ORBIT_SLOTS)-th of ORBIT_SEGS equal parts of the rows its rays cross; the parts' sums
// are added in a fixed order through shared memory.
template <typename S, bool NAMED = false, int SEGS = ORBIT_SEGS, int SLOTS = ORBIT_SLOTS, bool PAIRS = false>
__device__ __forceinline__ void forward_orbit_body(const typename OrbitRec<S>::type *__restrict__ ubar, int n,
                                                   int n_jobs, int M, const OrbitJob *__restrict__ jobs,
                                                   const ForwardEpi<float> &epi, int bx, int by)
{
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int slot = warp % SLOTS, seg = warp / SLOTS;
    const int jb = by * SLOTS + slot;
    const int kb = bx * 31;
    const int k = kb + lane - 1;
    const bool active = jb < n_jobs && kb < M;        // warp-uniform
    float4 Su = make_float4(0.f, 0.f, 0.f, 0.f), Sf = Su;
    int4 ls = make_int4(-1, -1, -1, -1);             // the job's angles
    __shared__ float s_epi[SLOTS][4 * 5 * 32];
    const bool pre = (epi.mode == 1 || epi.mode == 2) && seg == 0 && active;   // warp-uniform
    if (active) {
        const AngleMarch am = jobs[jb].am;
        ls = *reinterpret_cast<const int4 *>(jobs[jb].l);
        if (pre) orbit_epi_prefetch(epi, ls, M, k, lane, s_epi[slot]);
        const float Q0 = (float)k * am.kA - am.oA;
        int mlo, mhi;
        rows_in<true>(Q0, am.binv, -3.f, (float)n + 1.f, n, mlo, mhi);
        int mlo_w = __reduce_min_sync(0xffffffffu, mlo);
        int mhi_w = __reduce_max_sync(0xffffffffu, mhi);
        if (mlo_w <= mhi_w) {
            int ilo, ihi;
            rows_in<false>(Q0, am.binv, 0.5f, (float)n - 3.5f, n, ilo, ihi);
            int ilo_w = max(__reduce_max_sync(0xffffffffu, ilo), mlo_w);
            int ihi_w = min(__reduce_min_sync(0xffffffffu, ihi), mhi_w);
            if (SEGS > 1) {                     // this warp's part of the rows
                const int per = (mhi_w - mlo_w + SEGS) / SEGS;
                const int a = mlo_w + seg * per, b = min(mhi_w, a + per - 1);
                mlo_w = a;
                mhi_w = b;
                ilo_w = max(ilo_w, a);
                ihi_w = min(ihi_w, b);
            }
            if (mlo_w <= mhi_w) {
                const long long K = (long long)k << 32;
                // a pair job (channels {0, 1} or {2, 3} only; odd view counts give only these)
                // reads and accumulates its two live channels; the others stay zero as they
                // would in the four-channel march
                bool done = false;
                if constexpr (PAIRS && std::is_same<S, float>::value) {
                    const int pair = (ls.z < 0 && ls.w < 0) ? 1 : ((ls.x < 0 && ls.y < 0) ? 2 : 0);
                    if (pair) {
                        const PairLoad ld{reinterpret_cast<const float2 *>(ubar) + (pair - 1)};
                        float2 su = make_float2(0.f, 0.f), sf = su;
                        if (am.B > 0) march_orbit_rows<true>(ld, n, K, am, mlo_w, mhi_w, ilo_w, ihi_w, su, sf);
                        else march_orbit_rows<false>(ld, n, K, am, mlo_w, mhi_w, ilo_w, ihi_w, su, sf);
                        if (pair == 1) {
                            Su.x = su.x; Su.y = su.y; Sf.x = sf.x; Sf.y = sf.y;
                        } else {
                            Su.z = su.x; Su.w = su.y; Sf.z = sf.x; Sf.w = sf.y;
                        }
                        done = true;
                    }
                }
                if (!done) {
                    const RecLoad<typename OrbitRec<S>::type> ld{ubar};
                    if (am.B > 0) march_orbit_rows<true>(ld, n, K, am, mlo_w, mhi_w, ilo_w, ihi_w, Su, Sf);
                    else march_orbit_rows<false>(ld, n, K, am, mlo_w, mhi_w, ilo_w, ihi_w, Su, Sf);
                }
            }
        }
    }
    if constexpr (SEGS > 1) {
        __shared__ float4 s_part[SEGS > 1 ? SEGS - 1 : 1][2][SLOTS][32];
        if (seg > 0) {
            s_part[seg - 1][0][slot][lane] = Su;
            s_part[seg - 1][1][slot][lane] = Sf;
        }
        body_sync<NAMED>();
        if (seg > 0) return;
#pragma unroll
        for (int z = 0; z < SEGS - 1; ++z) {
            const float4 a = s_part[z][0][slot][lane], b = s_part[z][1][slot][lane];
            Su.x += a.x; Su.y += a.y; Su.z += a.z; Su.w += a.w;
            Sf.x += b.x; Sf.y += b.y; Sf.z += b.z; Sf.w += b.w;
        }
    }
    if (!active) return;
    if (pre) cp_async_wait<0>();                      // this lane's own copies: no barrier needed
    const float *pe = pre ? s_epi[slot] + lane : nullptr;
    orbit_out(epi, ls.x, M, k, lane, Su.x, Sf.x, pe ? pe + 0 * 160 : nullptr);
    orbit_out(epi, ls.y, M, k, lane, Su.y, Sf.y, pe ? pe + 1 * 160 : nullptr);
    orbit_out(epi, ls.z, M, k, lane, Su.z, Sf.z, pe ? pe + 2 * 160 : nullptr);
    orbit_out(epi, ls.w, M, k, lane, Su.w, Sf.w, pe ? pe + 3 * 160 : nullptr);
}

// SLOTS adjacent jobs per CTA (their rays nearly coincide, so they share the orbit
// image's lines in L1) and SEGS warps per job splitting its rows; the shape is selected per
// plan (ctr_plan_set_fwd_shape).  The resident-CTA hint keeps 32 warps per SM.
template <typename S, int SLOTS, int SEGS, bool PAIRS = false>
__global__ void __launch_bounds__(32 * SLOTS * SEGS, CTR_ORBIT_MINB * ORBIT_SLOTS * ORBIT_SEGS / (SLOTS * SEGS))
k_forward_orbit(const typename OrbitRec<S>::type *__restrict__ ubar, int n, int n_jobs, int M,
                const OrbitJob *__restrict__ jobs, ForwardEpi<float> epi)
{
    pdl_wait();
    pdl_trigger();
    forward_orbit_body<S, false, SEGS, SLOTS, PAIRS>(ubar, n, n_jobs, M, jobs, epi, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Symmetric forward projector with shared staging (launch shape (4, 1)).  A CTA takes
// STG_JOBS consecutive jobs -- adjacent canonical angles, whose rays nearly coincide --
// one warp each, and the same 31 bins.  All warps march the same rows; for every block of
// STG_ROWS rows the union of the jobs' bands of the orbit image (the pixels their rays
// cross there) is copied into shared memory with 16-byte cp.async (zero-filled outside the
// image) while the previous block is marched, so each pixel the group reads comes once from
// L2 for the four jobs instead of once per job.  Weights, march and sums are those of
// k_forward_orbit (one warp per job, no row split), so the results equal its shape (1, 1).
// The window of a block is the union over the jobs of [first pixel of interval kb - 1 on
// the block's last row, last pixel of interval kb + 30 on its first row]; the plan holds
// the widest window any block can need (stg_window), which sizes the row pitch.
// ---------------------------------------------------------------------------
constexpr int STG_JOBS = 4;
constexpr int STG_ROWS = 8;

template <typename R>
__device__ __forceinline__ void cp_async_rec(R *dst, const R *src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(R) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0)
                     : "memory");
}

template <typename S>
__global__ void __launch_bounds__(32 * STG_JOBS)
k_forward_orbit_staged(const typename OrbitRec<S>::type *__restrict__ ubar, int n, int n_jobs, int M,
                       const OrbitJob *__restrict__ jobs, ForwardEpi<float> epi, int wmax, int nst_max)
{
    using R = typename OrbitRec<S>::type;
    constexpr long long ONE = 4294967296ll;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *stage = reinterpret_cast<R *>(smem_raw);                        // [2][STG_ROWS][wmax]
    int *s_qlo = reinterpret_cast<int *>(stage + 2 * STG_ROWS * wmax);  // [nst_max]
    int *s_qhi = s_qlo + nst_max;
    __shared__ int s_mlo, s_mhi;
    pdl_wait();
    pdl_trigger();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kb = blockIdx.x * 31;
    const int k = kb + lane - 1;                 // this lane's interval [k, k + 1)
    const int j0 = blockIdx.y * STG_JOBS;
    const int nj = min(STG_JOBS, n_jobs - j0);
    const bool has_job = warp < nj;              // warp-uniform
    AngleMarch am{};
    int4 ls = make_int4(-1, -1, -1, -1);
    if (has_job) {
        am = jobs[j0 + warp].am;
        ls = *reinterpret_cast<const int4 *>(jobs[j0 + warp].l);
    }
    if (threadIdx.x == 0) {
        s_mlo = n;
        s_mhi = -1;
    }
    __syncthreads();
    {   // rows crossed by the CTA's rays on the detector (outer bounds, as k_forward_orbit)
        int mlo = n, mhi = -1;
        if (has_job && k < M) {
            const float Q0 = (float)k * am.kA - am.oA;
            rows_in<true>(Q0, am.binv, -3.f, (float)n + 1.f, n, mlo, mhi);
        }
        mlo = __reduce_min_sync(0xffffffffu, mlo);
        mhi = __reduce_max_sync(0xffffffffu, mhi);
        if (lane == 0 && mlo <= mhi) {
            atomicMin(&s_mlo, mlo);
            atomicMax(&s_mhi, mhi);
        }
    }
    __syncthreads();
    const int mlo = s_mlo, mhi = s_mhi;
    const int nst = mlo <= mhi ? min((mhi - mlo + STG_ROWS) / STG_ROWS, nst_max) : 0;
    for (int e = threadIdx.x; e < nst; e += blockDim.x) {
        s_qlo[e] = 0x7fffffff;
        s_qhi[e] = -0x7fffffff;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nst * nj; e += blockDim.x) {   // every block's window
        const int st = e / nj;
        const AngleMarch a = jobs[j0 + (e - st * nj)].am;
        const int mf = mlo + st * STG_ROWS, ml = min(mf + STG_ROWS - 1, mhi);
        const long long lo = ceil_div_ll((long long)(kb - 1) * ONE - (long long)ml * a.B - a.Op, a.A);
        const long long hi = ceil_div_ll((long long)(kb + 31) * ONE - (long long)mf * a.B - a.Op, a.A) - 1;
        atomicMin(&s_qlo[st], (int)lo);
        atomicMax(&s_qhi[st], (int)hi);
    }
    __syncthreads();
    // block st of rows into buffer st & 1: row rr at stage[(st & 1)][rr][c] = pixel q_lo + c
    auto prefetch = [&](int st) {
        R *dst = stage + (size_t)(st & 1) * STG_ROWS * wmax;
        const int q0 = s_qlo[st];
        const int w = min(s_qhi[st] - q0 + 1, wmax);
        const int mf = mlo + st * STG_ROWS;
        const int rows = min(STG_ROWS, mhi - mf + 1);
        for (int rr = 0; rr < rows; ++rr) {
            const R *src_row = ubar + (size_t)(mf + rr) * n;
            for (int c = threadIdx.x; c < w; c += blockDim.x) {
                const int q = q0 + c;
                const bool ok = (unsigned)q < (unsigned)n;
                cp_async_rec(dst + rr * wmax + c, ok ? src_row + q : ubar, ok);
            }
        }
    };
    float4 Su = make_float4(0.f, 0.f, 0.f, 0.f), Sf = Su;
    // the lane's march state at row mlo: q = first pixel with P >= K, r = P - K in [0, A)
    const long long A = am.A > 0 ? am.A : 1, B = am.B;
    const long long K = (long long)k * ONE;
    const long long qa = ceil_div_ll(K - (long long)mlo * B - am.Op, A);
    unsigned r = (unsigned)(qa * A + (long long)mlo * B + am.Op - K);
    int q = (int)qa;
    const unsigned A32 = (unsigned)A, B32 = (unsigned)B;
    const unsigned lim = (unsigned)(ONE - A);
    // the first pixel moves one to the left when r + B reaches A; with B = 0 it never moves
    // (and A - B may be 2^32, which a 32-bit threshold cannot hold)
    const unsigned thr = (unsigned)(A - B);
    const bool moves = B > 0;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    if (nst > 0) prefetch(0);
    cp_async_commit();
    for (int st = 0; st < nst; ++st) {
        if (st + 1 < nst) prefetch(st + 1);
        cp_async_commit();
        cp_async_wait<1>();                      // this thread's copies of block st
        __syncthreads();                         // everyone's
        if (has_job) {
            const R *blk = stage + (size_t)(st & 1) * STG_ROWS * wmax;
            const int rows = min(STG_ROWS, mhi - (mlo + st * STG_ROWS) + 1);
            int idx = q - s_qlo[st];
#pragma unroll
            for (int rr = 0; rr < STG_ROWS; ++rr) {
                if (rr < rows) {
                    const R *row = blk + rr * wmax;
                    const float4 v1 = rec_f32(row[idx]);
                    const float4 v2 = r < lim ? rec_f32(row[idx + 1]) : zero;
                    acc4(Su, Sf, v1, one_plus_frac32u(r));
                    acc4(Su, Sf, v2, one_plus_frac32u(r + A32));
                    const bool sdn = moves && r >= thr;
                    r += sdn ? B32 - A32 : B32;
                    idx -= sdn ? 1 : 0;
                    q -= sdn ? 1 : 0;
                }
            }
        }
        __syncthreads();                         // buffer st & 1 is refilled next
    }
    cp_async_wait<0>();
    if (!has_job || kb >= M) return;             // warp-uniform
    orbit_out(epi, ls.x, M, k, lane, Su.x, Sf.x);
    orbit_out(epi, ls.y, M, k, lane, Su.y, Sf.y);
    orbit_out(epi, ls.z, M, k, lane, Su.z, Sf.z);
    orbit_out(epi, ls.w, M, k, lane, Su.w, Sf.w);
}

template <typename S>
void launch_forward_orbit_staged(const ctr_plan *p, const typename OrbitRec<S>::type *ub,
                                 const ForwardEpi<float> &epi, cudaStream_t s)
{
    const dim3 grid(fwd_grid_x(p->M), (p->n_jobs + STG_JOBS - 1) / STG_JOBS);
    const int rec = (int)sizeof(typename OrbitRec<S>::type);
    launch_pdl(p->pdl != 0, k_forward_orbit_staged<S>, grid, dim3(32 * STG_JOBS),
               stg_smem_bytes(p->stg_wmax, p->stg_nst, rec), s, ub, p->n, p->n_jobs, p->M,
               (const OrbitJob *)p->d_jobs, epi, p->stg_wmax, p->stg_nst);
}

template <typename S, int SLOTS, int SEGS>
void launch_forward_orbit_shape(const ctr_plan *p, const typename OrbitRec<S>::type *ub, const ForwardEpi<float> &epi,
                                cudaStream_t s)
{
    const dim3 grid(fwd_grid_x(p->M), (p->n_jobs + SLOTS - 1) / SLOTS);
    auto kern = k_forward_orbit<S, SLOTS, SEGS, false>;
    if constexpr (std::is_same<S, float>::value)                  // pair-job variant (two live channels)
        if (p->pair_jobs) kern = k_forward_orbit<S, SLOTS, SEGS, true>;
    launch_pdl(p->pdl != 0, kern, grid, dim3(32 * SLOTS * SEGS), 0, s, ub, p->n, p->n_jobs, p->M,
               (const OrbitJob *)p->d_jobs, epi);
}

template <typename S>
void launch_forward_orbit(const ctr_plan *p, const typename OrbitRec<S>::type *ub, const ForwardEpi<float> &epi,
                          cudaStream_t s)
{
    switch (p->fwd_slots * 16 + p->fwd_segs) {
    case 1 * 16 + 2: launch_forward_orbit_shape<S, 1, 2>(p, ub, epi, s); break;
    case 1 * 16 + 8: launch_forward_orbit_shape<S, 1, 8>(p, ub, epi, s); break;
    case 2 * 16 + 2: launch_forward_orbit_shape<S, 2, 2>(p, ub, epi, s); break;
    case 2 * 16 + 4: launch_forward_orbit_shape<S, 2, 4>(p, ub, epi, s); break;
    case 4 * 16 + 2: launch_forward_orbit_shape<S, 4, 2>(p, ub, epi, s); break;
    case 4 * 16 + 1: launch_forward_orbit_staged<S>(p, ub, epi, s); break;
    default: launch_forward_orbit_shape<S, 1, 4>(p, ub, epi, s); break;
    }
}

// ---------------------------------------------------------------------------
// Symmetric backprojection (OrbitJob): a CTA owns a 32 x 32 tile of canonical
// pixels x and a group of jobs; per job it stages the four channels' sinogram rows
// side by side, so one fixed-point P(x) and one pair of 16-byte shared loads serve
// four angles.  Channel v's sum at x belongs to image pixel T_v^{-1}(x); the four
// channel images are written as partial planes [group][v][row][col] with
//   plane 0 at x, plane 1 at x (its pixel is row-mirrored), planes 2 and 3 transposed
// so that the fold reads rows only:
//   u(i, j) = sum_groups P0[i][j] + P1[n-1-i][j] + P2[i][j] + P3[n-1-i][j].
// ---------------------------------------------------------------------------
#ifndef CTR_OBP_TY
#define CTR_OBP_TY 8
#endif
#ifndef CTR_OBP_R
#define CTR_OBP_R 4
#endif
constexpr int OBP_TY = CTR_OBP_TY;     // warps of a symmetric-backprojection CTA (32 x 32 tile)
constexpr int OBP_R = CTR_OBP_R;       // pixels per thread (rows i0 + ty + OBP_TY r)
#ifndef CTR_OBP_ASYNC
#define CTR_OBP_ASYNC 1
#endif
constexpr bool OBP_ASYNC = CTR_OBP_ASYNC;
#ifndef CTR_OBP_JCH
#define CTR_OBP_JCH 8
#endif
constexpr int OBP_JCH = CTR_OBP_JCH;   // jobs per staged chunk (synchronous staging)
#ifndef CTR_OBP_AJCH
#define CTR_OBP_AJCH 24
#endif
constexpr int OBP_AJCH = CTR_OBP_AJCH; // jobs per staged chunk (asynchronous staging, two buffers)

size_t obp_smem(int wstride, int jobs_per_group)
{
    // staged pairs + chunk tables (bfloat16 operands, synchronous staging) ...
    const size_t stage = sizeof(float4) * 2 * OBP_JCH * wstride + (3 * sizeof(long long) + 5 * sizeof(int)) * OBP_JCH;
    // ... or two raw chunk buffers + the whole group's tables (FP32, asynchronous staging)
    const size_t async = sizeof(float4) * 2 * OBP_AJCH * (wstride + 1) +
                         (3 * sizeof(long long) + 5 * sizeof(int)) * (size_t)jobs_per_group;
    const size_t tr = sizeof(float) * 2 * 32 * 33;
    return std::max(std::max(stage, async), tr);
}

// The FP32 symmetric backprojection with asynchronous staging: the group's job tables
// are built once; chunk c + 1's four sinogram rows per job are copied raw into the
// second of two shared buffers (cp.async, zero-filled outside the detector) while
// chunk c is computed, so no global-load latency sits between chunks.  Each bin holds
// the four channels' g as one float4; a (pixel, job) reads bins b and b + 1 and
// interpolates g_b + f (g_{b+1} - g_b) per channel.
template <bool PAIRS>
__device__ __forceinline__ void obp_body_async(const float *__restrict__ g, int n, int M, int wstride,
                                               int jobs_per_group, int n_jobs, const OrbitJob *__restrict__ jobs,
                                               float (&acc)[OBP_R][4], int bx, int by, int bz)
{
    constexpr int NT = 32 * OBP_TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int WR = wstride + 1;                                           // bins per staged row
    float4 *raw = reinterpret_cast<float4 *>(smem_raw);                   // [2][JCH][WR], channels in x..w
    const int la = bz * jobs_per_group;
    const int nj = max(0, min(n_jobs, la + jobs_per_group) - la);
    // per job one 16-byte record {fraction of the tile's first P, S, C - 1, pair} (on the
    // symmetric path 0 <= S < 2^32 and 1 <= C <= 2^32; pair = 1 or 2 for a job whose angles
    // sit in channels {0, 1} or {2, 3} only, 0 otherwise): one shared load per warp and job
    uint4 *sT = reinterpret_cast<uint4 *>(raw + 2 * OBP_AJCH * WR);
    int *sK = reinterpret_cast<int *>(sT + jobs_per_group);
    int *sL = sK + jobs_per_group;                                        // [job][channel]
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int i0 = by * 32, j0 = bx * 32;
    for (int t = threadIdx.x; t < nj; t += NT) {
        const OrbitJob &jb = jobs[la + t];
        const long long Cc = jb.am.A, Sc = jb.am.B;
        const long long P00 = (long long)i0 * Cc + (long long)j0 * Sc + jb.am.Op;
        const long long kmin = P00 >> 32;                                // Cc, Sc >= 0: the tile's minimum
        sK[t] = (int)kmin;
        const unsigned pair = !PAIRS ? 0u : (jb.l[2] < 0 && jb.l[3] < 0) ? 1u : ((jb.l[0] < 0 && jb.l[1] < 0) ? 2u : 0u);
        sT[t] = make_uint4((unsigned)(P00 - (kmin << 32)), (unsigned)Sc, (unsigned)(Cc - 1), pair);
        for (int c = 0; c < 4; ++c) sL[4 * t + c] = jb.l[c];
    }
    __syncthreads();
    const int nch = (nj + OBP_AJCH - 1) / OBP_AJCH;
    auto prefetch = [&](int ch) {
        const int a0 = ch * OBP_AJCH, na = min(OBP_AJCH, nj - a0);
        float *dst = reinterpret_cast<float *>(raw + (size_t)(ch & 1) * OBP_AJCH * WR);
        // four-channel jobs: slot w = the four channels at bin k + w; pair jobs: slot w = the two
        // live channels at bins k + w and k + w + 1 (lo and hi of one interpolation)
        const unsigned mw = udiv_magic((unsigned)WR);
        for (int e = threadIdx.x; e < na * WR * 4; e += NT) {
            const int c = e & 3, rest = e >> 2;
            const int a = udiv_fast(rest, WR, mw), w = rest - a * WR;
            const unsigned pair = PAIRS ? sT[a0 + a].w : 0u;
            const int ch = pair ? 2 * (int)(pair - 1) + (c & 1) : c;
            const int k = sK[a0 + a] + w + (pair ? (c >> 1) : 0), l = sL[4 * (a0 + a) + ch];
            const bool ok = l >= 0 && k >= 0 && k < M;
            cp_async4(dst + (size_t)rest * 4 + c, ok ? g + (size_t)l * M + k : g, ok);
        }
    };
    if (nch > 0) prefetch(0);
    cp_async_commit();
    for (int ch = 0; ch < nch; ++ch) {
        if (ch + 1 < nch) prefetch(ch + 1);
        cp_async_commit();
        cp_async_wait<1>();                                               // this thread's copies of chunk ch
        __syncthreads();                                                  // everyone's
        const int a0 = ch * OBP_AJCH, na = min(OBP_AJCH, nj - a0);
        const float4 *buf = raw + (size_t)(ch & 1) * OBP_AJCH * WR;
#pragma unroll 2
        for (int a = 0; a < na; ++a) {
            const uint4 tj = sT[a0 + a];
            const long long C = (long long)tj.z + 1;
            long long P = (long long)tj.x + (long long)ty * C + (long long)tx * (long long)tj.y;
            const long long D = C * OBP_TY;
            const float4 *row = buf + a * WR;
            if (PAIRS && tj.w) {                                          // pair job (CTA-uniform)
                const bool p01 = tj.w == 1;
#pragma unroll
                for (int r = 0; r < OBP_R; ++r) {
                    const int b = (int)(P >> 32);
                    const float f = one_plus_frac32(P) - 1.f;
                    const float4 v = row[b];                              // (lo, lo, hi, hi)
                    const float2 lo = make_float2(v.x, v.y);
                    const float2 t = ffma2(make_float2(f, f), fsub2(make_float2(v.z, v.w), lo), lo);
                    if (p01) {
                        const float2 s = fadd2(make_float2(acc[r][0], acc[r][1]), t);
                        acc[r][0] = s.x;
                        acc[r][1] = s.y;
                    } else {
                        const float2 s = fadd2(make_float2(acc[r][2], acc[r][3]), t);
                        acc[r][2] = s.x;
                        acc[r][3] = s.y;
                    }
                    P += D;
                }
                continue;
            }
#pragma unroll
            for (int r = 0; r < OBP_R; ++r) {
                const int b = (int)(P >> 32);
                const float f = one_plus_frac32(P) - 1.f;                 // exact: the 23 fraction bits
                const float4 lo = row[b], hi = row[b + 1];
                const float2 f2 = make_float2(f, f);
                const float2 lo01 = make_float2(lo.x, lo.y), lo23 = make_float2(lo.z, lo.w);
                const float2 t01 = ffma2(f2, fsub2(make_float2(hi.x, hi.y), lo01), lo01);
                const float2 t23 = ffma2(f2, fsub2(make_float2(hi.z, hi.w), lo23), lo23);
                const float2 a01 = fadd2(make_float2(acc[r][0], acc[r][1]), t01);
                const float2 a23 = fadd2(make_float2(acc[r][2], acc[r][3]), t23);
                acc[r][0] = a01.x;
                acc[r][1] = a01.y;
                acc[r][2] = a23.x;
                acc[r][3] = a23.y;
                P += D;
            }
        }
        __syncthreads();                                                  // buffer ch & 1 is refilled next
    }
    cp_async_wait<0>();
}

template <typename S, bool PAIRS = false>
__device__ __forceinline__ void obp_body(const S *__restrict__ g, int n, int M, int wstride, int jobs_per_group,
                                         int n_jobs, const OrbitJob *__restrict__ jobs, float *__restrict__ part,
                                         int bx, int by, int bz)
{
    static_assert(OBP_TY * OBP_R == 32, "32 x 32 tiles");
    constexpr int NT = 32 * OBP_TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *stage = reinterpret_cast<float4 *>(smem_raw);               // [job][channel pair][bin]
    long long *sPb = reinterpret_cast<long long *>(stage + 2 * OBP_JCH * wstride);
    long long *sC = sPb + OBP_JCH;
    long long *sS = sC + OBP_JCH;
    int *sK = reinterpret_cast<int *>(sS + OBP_JCH);
    int *sL = sK + OBP_JCH;                                               // [job][channel]

    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int i0 = by * 32, j0 = bx * 32;
    const int la = bz * jobs_per_group;
    const int lb = min(n_jobs, la + jobs_per_group);
    float acc[OBP_R][4];
#pragma unroll
    for (int r = 0; r < OBP_R; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.f;

    if constexpr (sizeof(S) == 4 && OBP_ASYNC)
        obp_body_async<PAIRS>(g, n, M, wstride, jobs_per_group, n_jobs, jobs, acc, bx, by, bz);
    else
    for (int c0 = la; c0 < lb; c0 += OBP_JCH) {
        const int na = min(OBP_JCH, lb - c0);
        __syncthreads();
        if (threadIdx.x < na) {
            const AngleMarch am = jobs[c0 + threadIdx.x].am;     // canonical P(i, j) = i A + j B + Op
            const long long Cc = am.A, Sc = am.B;
            const long long P00 = (long long)i0 * Cc + (long long)j0 * Sc + am.Op;
            const long long kmin = P00 >> 32;                    // Cc, Sc >= 0: P00 is the tile's minimum
            sK[threadIdx.x] = (int)kmin;
            sPb[threadIdx.x] = P00 - (kmin << 32);
            sC[threadIdx.x] = Cc;
            sS[threadIdx.x] = Sc;
        }
        if (threadIdx.x < 4 * na) sL[threadIdx.x] = jobs[c0 + (threadIdx.x >> 2)].l[threadIdx.x & 3];
        __syncthreads();
        float *stf = reinterpret_cast<float *>(stage);
        const unsigned mw = udiv_magic((unsigned)wstride);
        for (int e = threadIdx.x; e < na * wstride * 4; e += NT) {
            const int c = e & 3, rest = e >> 2;
            const int a = udiv_fast(rest, wstride, mw), w = rest - a * wstride;
            const int k = sK[a] + w, l = sL[4 * a + c];
            const S *row = g + (size_t)(l < 0 ? 0 : l) * M;
            const float g0 = (l >= 0 && k >= 0 && k < M) ? ldv(row + k) : 0.f;
            const float g1 = (l >= 0 && k + 1 >= 0 && k + 1 < M) ? ldv(row + k + 1) : 0.f;
            // float4 planes (ch0 ch1) and (ch2 ch3) of the job, consecutive bins adjacent; in
            // each float4 the two channels' (g0 - d) first, then their d = g1 - g0
            const float2 st = make_stage(g0, g1);
            float *q = stf + ((size_t)(2 * a + (c >> 1)) * wstride + w) * 4 + (c & 1);
            q[0] = st.x;
            q[2] = st.y;
        }
        __syncthreads();
#pragma unroll 2
        for (int a = 0; a < na; ++a) {
            const long long C = sC[a];
            long long P = sPb[a] + (long long)ty * C + (long long)tx * sS[a];
            const long long D = C * OBP_TY;
            const float4 *row01 = stage + 2 * a * wstride;
            const float4 *row23 = row01 + wstride;
#pragma unroll
            for (int r = 0; r < OBP_R; ++r) {
                const int b = (int)(P >> 32);
                const float f = one_plus_frac32(P);
                const float4 s01 = row01[b], s23 = row23[b];
                const float2 f2 = make_float2(f, f);
                const float2 a01 = ffma2(f2, make_float2(s01.z, s01.w),
                                         fadd2(make_float2(acc[r][0], acc[r][1]), make_float2(s01.x, s01.y)));
                const float2 a23 = ffma2(f2, make_float2(s23.z, s23.w),
                                         fadd2(make_float2(acc[r][2], acc[r][3]), make_float2(s23.x, s23.y)));
                acc[r][0] = a01.x;
                acc[r][1] = a01.y;
                acc[r][2] = a23.x;
                acc[r][3] = a23.y;
                P += D;
            }
        }
    }

    const size_t nn = (size_t)n * n;
    float *pg = part + (size_t)bz * 4 * nn;
    const int j = j0 + tx;
#pragma unroll
    for (int r = 0; r < OBP_R; ++r) {
        const int i = i0 + ty + OBP_TY * r;
        if (i < n && j < n) {
            pg[(size_t)i * n + j] = acc[r][0];
            pg[nn + (size_t)i * n + j] = acc[r][1];
        }
    }
    // planes 2 and 3 transposed through shared memory (coalesced rows j)
    __syncthreads();
    float(*tr)[32][33] = reinterpret_cast<float(*)[32][33]>(smem_raw);
#pragma unroll
    for (int r = 0; r < OBP_R; ++r) {
        tr[0][ty + OBP_TY * r][tx] = acc[r][2];
        tr[1][ty + OBP_TY * r][tx] = acc[r][3];
    }
    __syncthreads();
    const int it = i0 + tx;
#pragma unroll
    for (int r = 0; r < OBP_R; ++r) {
        const int jl = ty + OBP_TY * r, jt = j0 + jl;
        if (it < n && jt < n) {
            pg[2 * nn + (size_t)jt * n + it] = tr[0][tx][jl];
            pg[3 * nn + (size_t)jt * n + it] = tr[1][tx][jl];
        }
    }
}

template <typename S, bool PAIRS>
__global__ void __launch_bounds__(32 * OBP_TY, CTR_OBP_MINB)
k_backproject_orbit(const S *__restrict__ g, int n, int M, int wstride, int jobs_per_group, int n_jobs,
                    const OrbitJob *__restrict__ jobs, float *__restrict__ part)
{
    pdl_wait();
    pdl_trigger();
    obp_body<S, PAIRS>(g, n, M, wstride, jobs_per_group, n_jobs, jobs, part, blockIdx.x, blockIdx.y, blockIdx.z);
}

// The fold of the symmetric backprojection's partial planes, then the
// backprojection epilogue (grid-stride over the pixels).
__global__ void __launch_bounds__(256)
k_bp_fold(const float *__restrict__ part, int groups, int n, BackprojEpi<float> epi)
{
    pdl_wait();
    pdl_trigger();
    const size_t nn = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const int i = pix_i(e, n), j = pix_j(e, n);
        bp_epilogue(epi, n, i, j, orbit_fold(part, groups, n, i, j));
    }
}

// Batched stages: block b of the launch belongs to the slice s with
// prefix[s] <= b < prefix[s+1]; the slice's parameters come from its SliceDesc.
__device__ __forceinline__ int find_slice(const int *__restrict__ prefix, int ns, int b)
{
    int lo = 0, hi = ns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(32 * BP_TY)
k_backproject_batch(const SliceDesc *__restrict__ sd, const int *__restrict__ prefix, int ns)
{
    const int s = find_slice(prefix, ns, blockIdx.x);
    const SliceDesc &d = sd[s];
    const int local = blockIdx.x - prefix[s];
    const int bx = local % d.bp_tiles_x, rest = local / d.bp_tiles_x;
    const int by = rest % d.bp_tiles_y, bz = rest / d.bp_tiles_y;
    bp_body<float, float>(d.y1, d.n, d.N, d.M, 32, d.wstride, d.per_group, d.geom, d.bpe,
                          d.bp_groups > 1 ? d.bp_part : nullptr, bx, by, bz);
}

__global__ void __launch_bounds__(32 * OBP_TY, CTR_OBP_MINB)
k_backproject_orbit_batch(const SliceDesc *__restrict__ sd, const int *__restrict__ prefix, int ns)
{
    const int s = find_slice(prefix, ns, blockIdx.x);
    const SliceDesc &d = sd[s];
    const int local = blockIdx.x - prefix[s];
    const int bx = local % d.bp_tiles_x, rest = local / d.bp_tiles_x;
    const int by = rest % d.bp_tiles_y, bz = rest / d.bp_tiles_y;
    if (d.pair_jobs) obp_body<float, true>(d.y1, d.n, d.M, d.wstride, d.per_group, d.n_jobs, d.jobs, d.bp_part, bx, by, bz);
    else obp_body<float, false>(d.y1, d.n, d.M, d.wstride, d.per_group, d.n_jobs, d.jobs, d.bp_part, bx, by, bz);
}

__global__ void __launch_bounds__(256)
k_orbit_image_batch(const SliceDesc *__restrict__ sd, const int *__restrict__ prefix, int ns)
{
    const int s = find_slice(prefix, ns, blockIdx.x);
    const SliceDesc &d = sd[s];
    const int local = blockIdx.x - prefix[s], tiles = (d.n + 31) / 32;
    orbit_image_body<float>(d.u, d.ubar, d.n, local % tiles, local / tiles);
}

__global__ void __launch_bounds__(ORBIT_THREADS, CTR_ORBIT_MINB)
k_forward_orbit_batch(const SliceDesc *__restrict__ sd, const int *__restrict__ prefix, int ns)
{
    const int s = find_slice(prefix, ns, blockIdx.x);
    const SliceDesc &d = sd[s];
    const int local = blockIdx.x - prefix[s];
    if (d.pair_jobs)
        forward_orbit_body<float, false, ORBIT_SEGS, ORBIT_SLOTS, true>(d.ubar, d.n, d.n_jobs, d.M, d.jobs, d.fwe,
                                                                       local % d.fwd_chunks, local / d.fwd_chunks);
    else
        forward_orbit_body<float>(d.ubar, d.n, d.n_jobs, d.M, d.jobs, d.fwe, local % d.fwd_chunks, local / d.fwd_chunks);
}

__global__ void __launch_bounds__(FWD_THREADS)
k_forward_batch(const SliceDesc *__restrict__ sd, const int *__restrict__ prefix, int ns)
{
    const int s = find_slice(prefix, ns, blockIdx.x);
    const SliceDesc &d = sd[s];
    const int local = blockIdx.x - prefix[s];
    fwd_body<float, float, 2, true>(d.u, d.uT, d.n, d.N, d.M, 32, d.march, d.fwe, local % d.fwd_chunks,
                                    local / d.fwd_chunks);
}

template <typename T>
__global__ void __launch_bounds__(256) k_transpose(const T *__restrict__ in, T *__restrict__ out, int n)
{
    __shared__ T tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int i = by + r, j = bx + threadIdx.x;
        if (i < n && j < n) tile[r][threadIdx.x] = in[(size_t)i * n + j];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int i = bx + r, j = by + threadIdx.x;
        if (i < n && j < n) out[(size_t)i * n + j] = tile[threadIdx.x][r];
    }
}

template <typename T>
size_t bp_smem(const ctr_plan *p)
{
    using T2 = typename Pair<T>::type;
    return sizeof(T2) * BP_ACH * p->wstride + 3 * sizeof(long long) * BP_ACH + sizeof(int) * BP_ACH;
}

template <typename T, typename S, int NC, bool EXACT1>
void launch_fwd_cfg(const ctr_plan *p, dim3 grid, const S *u, const S *uT, const ForwardEpi<T> &epi, cudaStream_t s)
{
    k_forward<T, S, NC, EXACT1><<<grid, FWD_THREADS, 0, s>>>(u, uT, p->n, p->N, p->M, p->F, p->d_march, epi);
}

template <typename T, typename S>
ctr_status bp_impl(const ctr_plan *p, const S *g, const BackprojEpi<T> &epi, cudaStream_t s, bool defer_reduce)
{
    if constexpr (sizeof(T) == 4) {
        if (p->orbit) {
            const int G = p->obp_groups;
            dim3 grid((p->n + BP_TJ - 1) / BP_TJ, (p->n + BP_TI - 1) / BP_TI, G);
            float *part = (float *)p->obp_part;
            p->launches++;
            const int jpg = (p->n_jobs + G - 1) / G;
            auto kern = k_backproject_orbit<S, false>;
            if constexpr (sizeof(S) == 4)                                 // pair-job variant: FP32 staging only
                if (p->pair_jobs) kern = k_backproject_orbit<S, true>;
            launch_pdl(p->pdl != 0, kern, grid, dim3(32 * OBP_TY), obp_smem(p->wstride, jpg), s,
                       g, p->n, p->M, p->wstride, jpg, p->n_jobs, (const OrbitJob *)p->d_jobs, part);
            CTR_CHECK_LAUNCH("k_backproject_orbit");
            if (!defer_reduce) {
                const size_t nn = (size_t)p->n * p->n;
                int blocks = (int)((nn + 255) / 256);
                if (blocks > 4096) blocks = 4096;
                p->launches++;
                launch_pdl(p->pdl != 0, k_bp_fold, dim3(blocks), dim3(256), 0, s, (const float *)part, G, p->n, epi);
                CTR_CHECK_LAUNCH("k_bp_fold");
            }
            return CTR_OK;
        }
    }
    const int G = p->bp_groups;
    const int per = (p->N + G - 1) / G;
    dim3 grid((p->n + BP_TJ - 1) / BP_TJ, (p->n + BP_TI - 1) / BP_TI, G);
    T *part = G > 1 ? (T *)p->bp_part : nullptr;
    p->launches++;
    k_backproject<T, S><<<grid, 32 * BP_TY, bp_smem<T>(p), s>>>(g, p->n, p->N, p->M, p->F, p->wstride, per,
                                                                 p->d_geom, epi, part);
    CTR_CHECK_LAUNCH("k_backproject");
    if (G > 1 && !defer_reduce) {
        const size_t nn = (size_t)p->n * p->n;
        int blocks = (int)((nn + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        p->launches++;
        k_bp_reduce<T><<<blocks, 256, 0, s>>>(part, G, p->n, epi);
        CTR_CHECK_LAUNCH("k_bp_reduce");
    }
    return CTR_OK;
}

template <typename T, typename S>
ctr_status fwd_impl(const ctr_plan *p, const S *u, const S *uT, const ForwardEpi<T> &epi, cudaStream_t s,
                    const TvDualJob<T> *tv = nullptr)
{
    const bool exact1 = p->h <= p->ds;
    if constexpr (sizeof(T) == 4) {
        if (p->orbit) {
            using R = typename OrbitRec<S>::type;
            R *ub = (R *)p->ubar;
            p->launches++;
            const dim3 og((p->n + 31) / 32, (p->n + 31) / 32);
            if constexpr (std::is_same<S, float>::value) {
                if (tv) launch_pdl(p->pdl != 0, k_orbit_image_tv, og, dim3(256), 0, s, u, ub, p->n, *tv);
                else launch_pdl(p->pdl != 0, k_orbit_image<S>, og, dim3(256), 0, s, u, ub, p->n);
            } else {
                launch_pdl(p->pdl != 0, k_orbit_image<S>, og, dim3(256), 0, s, u, ub, p->n);
            }
            CTR_CHECK_LAUNCH("k_orbit_image");
            p->launches++;
            launch_forward_orbit<S>(p, ub, epi, s);
            CTR_CHECK_LAUNCH("k_forward_orbit");
            return CTR_OK;
        }
    }
    p->launches++;
    dim3 grid(fwd_grid_x(p->M), fwd_grid_y(p->N));
    switch (p->ncand * 2 + (exact1 ? 1 : 0)) {
    case 2: launch_fwd_cfg<T, S, 1, false>(p, grid, u, uT, epi, s); break;
    case 3: launch_fwd_cfg<T, S, 1, true>(p, grid, u, uT, epi, s); break;
    case 4: launch_fwd_cfg<T, S, 2, false>(p, grid, u, uT, epi, s); break;
    case 5: launch_fwd_cfg<T, S, 2, true>(p, grid, u, uT, epi, s); break;
    case 6: launch_fwd_cfg<T, S, 3, false>(p, grid, u, uT, epi, s); break;
    case 7: launch_fwd_cfg<T, S, 3, true>(p, grid, u, uT, epi, s); break;
    case 8: launch_fwd_cfg<T, S, 4, false>(p, grid, u, uT, epi, s); break;
    case 9: launch_fwd_cfg<T, S, 4, true>(p, grid, u, uT, epi, s); break;
    default: return fail(CTR_EUNSUPPORTED, "forward projector: too many pixels per detector interval");
    }
    CTR_CHECK_LAUNCH("k_forward");
    return CTR_OK;
}

}  // namespace

template <typename T>
ctr_status configure_radon(const ctr_plan *p)
{
    const size_t smem = bp_smem<T>(p);
    ctr_status st = raise_smem_limit(k_backproject<T, T>, smem);
    const size_t osm = p->orbit ? obp_smem(p->wstride, p->n_jobs) : 0;   // any group split
    if (st == CTR_OK && p->orbit) st = raise_smem_limit(k_backproject_orbit<float, false>, osm);
    if (st == CTR_OK && p->orbit) st = raise_smem_limit(k_backproject_orbit<float, true>, osm);
    if (st == CTR_OK && p->orbit) st = raise_smem_limit(k_backproject_orbit<__nv_bfloat16, false>, osm);
    if constexpr (sizeof(T) == 4)
        if (st == CTR_OK) st = raise_smem_limit(k_backproject<float, __nv_bfloat16>, smem);
    if (st == CTR_OK && p->orbit && p->stg_wmax > 0) {
        st = raise_smem_limit(k_forward_orbit_staged<float>, stg_smem_bytes(p->stg_wmax, p->stg_nst, 16));
        if (st == CTR_OK)
            st = raise_smem_limit(k_forward_orbit_staged<__nv_bfloat16>, stg_smem_bytes(p->stg_wmax, p->stg_nst, 8));
    }
    return st;
}

ctr_status launch_backproject_bf16(const ctr_plan *p, const __nv_bfloat16 *g, const BackprojEpi<float> &epi,
                                   cudaStream_t s, bool defer_reduce)
{
    return bp_impl<float, __nv_bfloat16>(p, g, epi, s, defer_reduce);
}

ctr_status launch_forward_bf16(const ctr_plan *p, const __nv_bfloat16 *u, const __nv_bfloat16 *uT,
                               const ForwardEpi<float> &epi, cudaStream_t s)
{
    return fwd_impl<float, __nv_bfloat16>(p, u, uT, epi, s);
}

template <typename T>
ctr_status launch_backproject(const ctr_plan *p, const T *g, const BackprojEpi<T> &epi, cudaStream_t s,
                              bool defer_reduce)
{
    return bp_impl<T, T>(p, g, epi, s, defer_reduce);
}

template <typename T>
ctr_status launch_forward(const ctr_plan *p, const T *u, const T *uT, const ForwardEpi<T> &epi, cudaStream_t s,
                          const TvDualJob<T> *tv)
{
    return fwd_impl<T, T>(p, u, uT, epi, s, tv);
}

template <typename T>
ctr_status launch_transpose(const ctr_plan *p, const T *in, T *out, cudaStream_t s)
{
    dim3 grid((p->n + 31) / 32, (p->n + 31) / 32);
    p->launches++;
    k_transpose<T><<<grid, dim3(32, 8), 0, s>>>(in, out, p->n);
    CTR_CHECK_LAUNCH("k_transpose");
    return CTR_OK;
}

int backproject_tile_rows() { return BP_TI; }

template <typename T>
bool bp_deferred(const ctr_plan *p)
{
    return p->bp_groups > 1 || (sizeof(T) == 4 && p->orbit);
}
template bool bp_deferred<float>(const ctr_plan *);
template bool bp_deferred<double>(const ctr_plan *);

int fwd_grid_x(int M) { return (M + 30) / 31; }

size_t stg_smem_bytes(int wmax, int nst_max, int rec_bytes)
{
    return (size_t)2 * STG_ROWS * wmax * rec_bytes + 2 * sizeof(int) * (size_t)nst_max;
}

int stg_blocks_max(int n) { return (n + STG_ROWS) / STG_ROWS + 1; }

// The widest window a staged block can need, over every group of STG_JOBS consecutive jobs:
// the spread of the jobs' first pixels at equal (K, m) (linear in K and m for each job, so
// its extremes lie at the corners of the detector x row range) plus the pixels 32 intervals
// and STG_ROWS - 1 rows span for the steepest job, plus the rounding of both window ends.
int stg_window(const std::vector<OrbitJob> &jobs, int n, int M)
{
    const double one = 4294967296.0;
    double w = 0.0;
    for (size_t g = 0; g < jobs.size(); g += STG_JOBS) {
        const size_t e = std::min(jobs.size(), g + STG_JOBS);
        double spread = 0.0, span = 0.0;
        for (double K : {-one, (double)(M + 32) * one})
            for (double m : {0.0, (double)(n - 1)}) {
                double lo = 1e300, hi = -1e300;
                for (size_t j = g; j < e; ++j) {
                    const double x = (K - m * (double)jobs[j].am.B - (double)jobs[j].am.Op) / (double)jobs[j].am.A;
                    lo = std::min(lo, x);
                    hi = std::max(hi, x);
                }
                spread = std::max(spread, hi - lo);
            }
        for (size_t j = g; j < e; ++j)
            span = std::max(span, (32.0 * one + (STG_ROWS - 1) * (double)jobs[j].am.B) / (double)jobs[j].am.A);
        w = std::max(w, std::ceil(spread + span) + 4.0);
    }
    return (int)w;
}

int orbit_fwd_grid_y(int n_jobs) { return (n_jobs + ORBIT_SLOTS - 1) / ORBIT_SLOTS; }
int fwd_grid_y(int N) { return (N + FWD_AW - 1) / FWD_AW; }

size_t obp_smem_bytes(int wstride, int jobs_per_group) { return obp_smem(wstride, jobs_per_group); }

size_t bp_smem_bytes(int wstride)
{
    return sizeof(float2) * BP_ACH * wstride + 3 * sizeof(long long) * BP_ACH + sizeof(int) * BP_ACH;
}

void bp_tiles(int n, int &tx, int &ty)
{
    tx = (n + BP_TJ - 1) / BP_TJ;
    ty = (n + BP_TI - 1) / BP_TI;
}

ctr_status configure_batch_radon(size_t bp_smem, size_t obp_smem_max)
{
    ctr_status st = raise_smem_limit(k_backproject_batch, bp_smem);
    if (st == CTR_OK) st = raise_smem_limit(k_backproject_orbit_batch, obp_smem_max);
    return st;
}

// One batched projector stage over all slices (blocks = total CTAs of the stage).
ctr_status launch_batch_radon(int stage, const SliceDesc *sd, const int *prefix, int ns, int blocks, size_t smem,
                              cudaStream_t s)
{
    if (blocks <= 0) return CTR_OK;
    switch (stage) {
    case BS_BP: k_backproject_batch<<<blocks, 32 * BP_TY, smem, s>>>(sd, prefix, ns); break;
    case BS_BP_SYM: k_backproject_orbit_batch<<<blocks, 32 * OBP_TY, smem, s>>>(sd, prefix, ns); break;
    case BS_ORBIT: k_orbit_image_batch<<<blocks, 256, 0, s>>>(sd, prefix, ns); break;
    case BS_FWD_SYM: k_forward_orbit_batch<<<blocks, ORBIT_THREADS, 0, s>>>(sd, prefix, ns); break;
    case BS_FWD: k_forward_batch<<<blocks, FWD_THREADS, 0, s>>>(sd, prefix, ns); break;
    default: return fail(CTR_EINVAL, "not a projector stage");
    }
    CTR_CHECK_LAUNCH("batched projector stage");
    return CTR_OK;
}

template ctr_status launch_backproject<float>(const ctr_plan *, const float *, const BackprojEpi<float> &, cudaStream_t,
                                             bool);
template ctr_status launch_backproject<double>(const ctr_plan *, const double *, const BackprojEpi<double> &,
                                              cudaStream_t, bool);
template ctr_status launch_forward<float>(const ctr_plan *, const float *, const float *, const ForwardEpi<float> &,
                                         cudaStream_t, const TvDualJob<float> *);
template ctr_status launch_forward<double>(const ctr_plan *, const double *, const double *,
                                          const ForwardEpi<double> &, cudaStream_t, const TvDualJob<double> *);
template ctr_status configure_radon<float>(const ctr_plan *);
template ctr_status configure_radon<double>(const ctr_plan *);
template ctr_status launch_transpose<float>(const ctr_plan *, const float *, float *, cudaStream_t);
template ctr_status launch_transpose<double>(const ctr_plan *, const double *, double *, cudaStream_t);
template ctr_status launch_transpose<__nv_bfloat16>(const ctr_plan *, const __nv_bfloat16 *, __nv_bfloat16 *, cudaStream_t);

}  // namespace ctr
