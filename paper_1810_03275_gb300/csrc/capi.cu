// The C ABI of libctrecon (declared in include/ctrecon.h): argument checking,
// plan construction (fixed-point geometry tables, FFT plan, device workspace),
// dtype dispatch and stream handling.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <utility>

#include "ctr_internal.cuh"

namespace ctr {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

ctr_status fail(ctr_status st, const std::string &msg)
{
    set_error(msg);
    return st;
}

ctr_status cuda_fail(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return CTR_ECUDA;
}

// implemented in solver.cu
template <typename T> ctr_status dot2(ctr_plan *, const T *, const T *, size_t, double *, cudaStream_t);
template <typename T> ctr_status op_grad(ctr_plan *, const T *, T *, cudaStream_t);
template <typename T> ctr_status op_div(ctr_plan *, const T *, T *, cudaStream_t);
template <typename T> ctr_status op_forward(ctr_plan *, const T *, const T *, T *, double, cudaStream_t);
template <typename T> ctr_status op_adjoint(ctr_plan *, const T *, T *, double, cudaStream_t);
ctr_status batch_solve(ctr_batch *, const float *const *, const uint8_t *const *, const double *, const double *, int,
                       const ctr_params &, const double *, const double *, float *const *, ctr_diag *, cudaStream_t);
ctr_status batch_prepare(ctr_batch *);
template <typename T>
ctr_status pdrq_vjp_step(ctr_plan *, const T *, const T *, const T *, const T *, const T *, const T *, const uint8_t *,
                         double, double, double, double, double, const ctr_params &, T *, T *, T *, T *, double *,
                         cudaStream_t);
ctr_status op_forward_bf16(ctr_plan *, const __nv_bfloat16 *, const __nv_bfloat16 *, float *, cudaStream_t);
ctr_status op_adjoint_bf16(ctr_plan *, const __nv_bfloat16 *, float *, cudaStream_t);
template <typename T> ctr_status power_beta(ctr_plan *, int, double *, cudaStream_t);
template <typename T> ctr_status power_lambda(ctr_plan *, double, double, int, double *, cudaStream_t);
template <typename T>
ctr_status pdrq_loop(ctr_plan *, double, int, const ctr_params &, double, double, ctr_diag *, cudaStream_t);
template <typename T>
ctr_status cp_loop(ctr_plan *, double, int, const ctr_params &, double, double, double, ctr_diag *, cudaStream_t);
template <typename T> ctr_status prepare_impulse_symbol(ctr_plan *, cudaStream_t);
template <typename T>
ctr_status admm_loop(ctr_plan *, double, int, int, double, const ctr_params &, double, double, ctr_diag *,
                     cudaStream_t);
template <typename T>
ctr_status metal_trace(ctr_plan *, const T *, double, int, double, uint8_t *, uint8_t *, cudaStream_t);

// The preconditioner that params select (inverse norm, impulse response, circulant or
// Richardson); the DFTs of the impulse-response and circulant kernels are built on their
// first use by the plan.
template <typename T>
ctr_status select_precond(ctr_plan *p, const ctr_params &q, cudaStream_t s)
{
    p->precond_kind = q.precond;
    return (q.precond == 1 || q.precond == 2) ? prepare_impulse_symbol<T>(p, s) : CTR_OK;
}
template <typename T>
ctr_status build_desc_from_data(ctr_plan *, const T *, const uint8_t *, double, double, double, cudaStream_t);
template <typename T>
ctr_status build_desc_from_arrays(ctr_plan *, const T *, const T *, const T *, const T *, double, cudaStream_t);

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

ctr_status alloc(ctr_plan *p, void **ptr, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(CTR_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    }
    p->allocations.push_back(*ptr);
    p->bytes += bytes;
    return CTR_OK;
}

long long floor_div2(__int128 v)
{
    __int128 q = v / 2;
    if (q * 2 > v) --q;
    return (long long)q;
}

// Groups the angles of an FP32 plan into the forward projector's symmetric jobs
// (OrbitJob): every angle's (C, S) must be one of (a, b), (-a, b), (b, a), (-b, a) of
// its canonical pair a = max(|C|, |S|), b = min(|C|, |S|) (true for angles in
// [0, pi)); angles with equal canonical pairs share a job, one per channel.  The
// path is taken when the jobs hold two angles or more on average.
ctr_status build_orbit_jobs(ctr_plan *p, const std::vector<AngleGeom> &geo)
{
    const int n = p->n, N = p->N, M = p->M;
    std::vector<OrbitJob> jobs;
    std::map<std::pair<long long, long long>, std::vector<int>> by_pair;   // canonical pair -> jobs
    for (int l = 0; l < N; ++l) {
        const long long C = geo[l].C, S = geo[l].S;
        const long long aC = C < 0 ? -C : C, aS = S < 0 ? -S : S;
        const long long a = aC >= aS ? aC : aS, b = aC >= aS ? aS : aC;
        // the symmetric kernels track 32-bit remainders and step at most one bin per row:
        // 1 <= a <= 2^32 (h <= ds makes it so; anything else takes the per-angle path)
        if (a < 1 || a > (1ll << 32)) return CTR_OK;
        const long long img[4][2] = {{a, b}, {-a, b}, {b, a}, {-b, a}};
        bool placed = false, member = false;
        std::vector<int> &js = by_pair[{a, b}];
        for (int v = 0; v < 4 && !placed; ++v) {
            if (img[v][0] != C || img[v][1] != S) continue;
            member = true;
            for (int j : js)
                if (jobs[j].l[v] < 0) {
                    jobs[j].l[v] = l;
                    placed = true;
                    break;
                }
        }
        if (!member) return CTR_OK;                 // outside the symmetric set: per-angle path
        if (!placed) {
            OrbitJob jb{};
            for (int v = 0; v < 4; ++v) jb.l[v] = -1;
            AngleMarch &am = jb.am;
            am.layout = 0;
            am.flip = 0;
            am.A = a;
            am.B = b;
            am.Op = floor_div2(((__int128)(M - 1) << 32) - (__int128)(n - 1) * ((__int128)a + (__int128)b));
            am.kA = (float)(4294967296.0 / (double)a);
            am.oA = (float)((double)am.Op / (double)a);
            const double bA = (double)b / (double)a;
            am.binv = bA > 1e-9 ? (float)(1.0 / bA) : 0.f;
            for (int v = 0; v < 4; ++v)
                if (img[v][0] == C && img[v][1] == S) { jb.l[v] = l; break; }
            js.push_back((int)jobs.size());
            jobs.push_back(jb);
        }
    }
    // at least two angles per job on average; an odd view count pairs every angle but 0 with
    // its mirror pi - theta ((N + 1) / 2 jobs), which the pair-job kernels serve at half cost
    if (2 * jobs.size() > (size_t)N + 1) return CTR_OK;
    ctr_status st;
    void *tmp = nullptr;
    if ((st = alloc(p, &tmp, sizeof(OrbitJob) * jobs.size())) != CTR_OK) return st;
    p->d_jobs = (OrbitJob *)tmp;
    if ((st = alloc(p, &p->ubar, sizeof(float4) * (size_t)n * n)) != CTR_OK) return st;
    // (the orbit image holds FP32 records; a BF16 plan's bfloat16 records use its first half)
    // the symmetric backprojection: job groups so that tiles x groups is about 1024 CTAs
    // (~1.7 waves of 4 eight-warp CTAs per SM on 152 SMs; measured best at n = 512 among
    // 2..8), at least 8 jobs per group; room for up to MAX_BP_GROUPS groups at n <= 1024
    // so that ctr_plan_set_bp_groups can change the split later
    const int tiles = ((n + 31) / 32) * ((n + 31) / 32);
    int G = (1024 + tiles / 2) / tiles;
    if (G > MAX_BP_GROUPS) G = MAX_BP_GROUPS;
    const int gmax = (int)jobs.size() / 8 > 1 ? (int)jobs.size() / 8 : 1;
    p->obp_groups = G > gmax ? gmax : (G < 1 ? 1 : G);
    p->obp_cap = n <= 1024 ? (gmax < MAX_BP_GROUPS ? gmax : MAX_BP_GROUPS) : p->obp_groups;
    if (p->obp_cap < p->obp_groups) p->obp_cap = p->obp_groups;
    if ((st = alloc(p, &p->obp_part, sizeof(float) * 4 * (size_t)p->obp_cap * n * n)) != CTR_OK) return st;
    CTR_CUDA(cudaMemcpy(p->d_jobs, jobs.data(), sizeof(OrbitJob) * jobs.size(), cudaMemcpyHostToDevice));
    p->n_jobs = (int)jobs.size();
    p->orbit = true;
    {
        size_t pairs = 0;                          // jobs whose angles sit in channels {0, 1} or {2, 3} only
        for (const OrbitJob &jb : jobs)
            if ((jb.l[2] < 0 && jb.l[3] < 0) || (jb.l[0] < 0 && jb.l[1] < 0)) ++pairs;
        p->pair_jobs = 2 * pairs > jobs.size() ? 1 : 0;
    }
    // the staged forward shape only where its double-buffered window fits one CTA's shared
    // memory (stg_wmax = 0: shape (4, 1) unavailable on this plan)
    p->stg_wmax = stg_window(jobs, n, M);
    p->stg_nst = stg_blocks_max(n);
    if (stg_smem_bytes(p->stg_wmax, p->stg_nst, 16) > STG_SMEM_LIMIT) p->stg_wmax = 0;
    return CTR_OK;
}

ctr_status build_tables(ctr_plan *p)
{
    const int n = p->n, N = p->N, M = p->M;
    std::vector<AngleGeom> geo(N);
    std::vector<AngleMarch> mar(N);
    const double ratio = p->h / p->ds;
    const long long one = 1ll << p->F;
    long long wmax = 0;
    int ncand = 1;
    for (int l = 0; l < N; ++l) {
        const double th = p->theta[l];
        const long long C = llround(ldexp(ratio * cos(th), p->F));
        const long long S = llround(ldexp(ratio * sin(th), p->F));
        // O: P(i, j) = i C + j S + O with p = (x_i cos + y_j sin)/ds + (M-1)/2, x_i = h(i - (n-1)/2)
        const __int128 num = ((__int128)(M - 1) << p->F) - (__int128)(n - 1) * ((__int128)C + (__int128)S);
        const long long O = floor_div2(num);
        geo[l] = AngleGeom{C, S, O};
        const long long aC = C < 0 ? -C : C, aS = S < 0 ? -S : S;
        if (aC == 0 && aS == 0) return fail(CTR_EINVAL, "degenerate geometry (h/ds too small)");
        // a backprojection tile spans (rows-1)|C| + 31|S| of P: its footprint in bins
        const long long w = (((long long)(backproject_tile_rows() - 1) * aC + 31 * aS) >> p->F) + 2;
        if (w > wmax) wmax = w;
        AngleMarch am{};
        if (aC >= aS) {
            am.layout = 0;   // pick along i (x), march along j
            if (C > 0) { am.A = C; am.Op = O; am.flip = 0; }
            else { am.A = -C; am.Op = O + (long long)(n - 1) * C; am.flip = 1; }
            am.B = S;
        } else {
            am.layout = 1;   // pick along j (y), march along i
            if (S > 0) { am.A = S; am.Op = O; am.flip = 0; }
            else { am.A = -S; am.Op = O + (long long)(n - 1) * S; am.flip = 1; }
            am.B = C;
        }
        am.kA = (float)((double)one / (double)am.A);
        am.oA = (float)((double)am.Op / (double)am.A);
        const double bA = (double)am.B / (double)am.A;
        am.binv = fabs(bA) > 1e-9 ? (float)(1.0 / bA) : 0.f;
        mar[l] = am;
        const long long nc = (one + am.A - 1) / am.A;
        if (nc > ncand) ncand = (int)nc;
    }
    if (ncand > 4) return fail(CTR_EUNSUPPORTED, "ds/h too large for the ray-driven projector (more than 4 pixels per bin and row)");
    p->ncand = ncand;
    p->wstride = (int)wmax;
    CTR_CUDA(cudaMemcpy(p->d_geom, geo.data(), sizeof(AngleGeom) * N, cudaMemcpyHostToDevice));
    CTR_CUDA(cudaMemcpy(p->d_march, mar.data(), sizeof(AngleMarch) * N, cudaMemcpyHostToDevice));
    if (p->F == 32 && p->h <= p->ds && ncand == 2) return build_orbit_jobs(p, geo);
    return CTR_OK;
}

template <typename T>
ctr_status build_twiddles(ctr_plan *p)
{
    const int n = p->n;
    std::vector<T> tw(2 * (size_t)n);
    const double pi = 3.14159265358979323846;
    for (int t = 0; t < n; ++t) {
        tw[2 * t] = (T)cos(2.0 * pi * t / n);
        tw[2 * t + 1] = (T)(-sin(2.0 * pi * t / n));
    }
    CTR_CUDA(cudaMemcpy(p->d_twiddle, tw.data(), sizeof(T) * tw.size(), cudaMemcpyHostToDevice));
    return CTR_OK;
}

void destroy(ctr_plan *p)
{
    if (!p) return;
    for (void *a : p->allocations) cudaFree(a);
    if (p->stream) cudaStreamDestroy(p->stream);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_out) cudaEventDestroy(p->ev_out);
    delete p;
}

ctr_status check_params(const ctr_params &q)
{
    if (!(q.sigma > 0) || !(q.tau > 0) || !std::isfinite(q.sigma) || !std::isfinite(q.tau))
        return fail(CTR_EINVAL, "sigma and tau must be finite and > 0");
    if (!(q.eps > 0) || !std::isfinite(q.eps)) return fail(CTR_EINVAL, "eps must be finite and > 0");
    if (!std::isfinite(q.c) || !std::isfinite(q.beta)) return fail(CTR_EINVAL, "c and beta must be finite");
    if (q.power_iters < 1) return fail(CTR_EINVAL, "power_iters must be >= 1");
    if (!(q.c_margin >= 1.0)) return fail(CTR_EINVAL, "c_margin must be >= 1");
    if (!std::isfinite(q.trace_ratio)) return fail(CTR_EINVAL, "trace_ratio must be finite");
    if (q.graph_block < 0 || q.check_every < 0) return fail(CTR_EINVAL, "graph_block and check_every must be >= 0");
    if (!(q.stop_tol >= 0) || !std::isfinite(q.stop_tol)) return fail(CTR_EINVAL, "stop_tol must be finite and >= 0");
    if (q.stop_tol > 0 && q.check_every < 1) return fail(CTR_EINVAL, "stop_tol > 0 needs check_every >= 1");
    if (q.nonneg != 0 && q.nonneg != 1) return fail(CTR_EINVAL, "nonneg must be 0 or 1");
    if (q.precond < 0 || q.precond > 3) return fail(CTR_EINVAL, "precond must be 0, 1, 2 or 3");
    return CTR_OK;
}

ctr_params resolve(const ctr_plan *p, const ctr_params *prm)
{
    ctr_params q;
    ctr_default_params(&q);
    if (prm) q = *prm;
    if (!(q.eps > 0)) q.eps = 3.14159265358979323846 / p->n;
    return q;
}

// Join the caller's stream to the plan's internal stream and back.
struct StreamJoin {
    ctr_plan *p;
    cudaStream_t user;
    bool joined = false;
    StreamJoin(ctr_plan *pp, void *s) : p(pp), user((cudaStream_t)s) {}
    ctr_status begin()
    {
        CTR_CUDA(cudaEventRecord(p->ev_in, user));
        CTR_CUDA(cudaStreamWaitEvent(p->stream, p->ev_in, 0));
        joined = true;
        return CTR_OK;
    }
    ~StreamJoin()
    {
        if (joined) {
            cudaEventRecord(p->ev_out, p->stream);
            cudaStreamWaitEvent(user, p->ev_out, 0);
        }
    }
};

template <typename T>
ctr_status solve_impl(ctr_plan *p, const void *f, const uint8_t *mask, const void *w, const void *a, const void *lo,
                      const void *hi, double alpha, double delta, int iters, const ctr_params &q, ctr_state *state,
                      void *u_out, ctr_diag *diag, void *stream)
{
    StreamJoin sj(p, stream);
    ctr_status st = sj.begin();
    if (st != CTR_OK) return st;
    cudaStream_t s = p->stream;
    if ((st = select_precond<T>(p, q, s)) != CTR_OK) return st;
    double beta = q.beta;
    if (!(beta > 0)) {
        if ((st = power_beta<T>(p, q.power_iters, &beta, s)) != CTR_OK) return st;
        if (!(beta > 0)) return fail(CTR_ENUMERIC, "power iteration gave ||R_h|| = 0");
    }
    double c = q.c;
    if (!(c > 0)) {
        double lam = 0;
        if ((st = power_lambda<T>(p, beta, q.eps, q.power_iters, &lam, s)) != CTR_OK) return st;
        c = q.c_margin * lam;
        if (!(c > 0)) return fail(CTR_ENUMERIC, "power iteration gave c <= 0");
    }
    if (f) st = build_desc_from_data<T>(p, (const T *)f, mask, delta, q.trace_ratio, beta, s);
    else st = build_desc_from_arrays<T>(p, (const T *)w, (const T *)a, (const T *)lo, (const T *)hi, beta, s);
    if (st != CTR_OK) return st;
    const size_t nn = (size_t)p->n * p->n, nm = (size_t)p->N * p->M;
    if (state) {
        CTR_CUDA(cudaMemcpyAsync(p->u, state->u, nn * sizeof(T), cudaMemcpyDeviceToDevice, s));
        CTR_CUDA(cudaMemcpyAsync(p->Ru, state->Ru, nm * sizeof(T), cudaMemcpyDeviceToDevice, s));
        CTR_CUDA(cudaMemcpyAsync(p->v1b, state->v1b, nm * sizeof(T), cudaMemcpyDeviceToDevice, s));
        CTR_CUDA(cudaMemcpyAsync(p->v2b, state->v2b, 2 * nn * sizeof(T), cudaMemcpyDeviceToDevice, s));
        if (q.nonneg) CTR_CUDA(cudaMemcpyAsync(p->ubar_u, state->ub, nn * sizeof(T), cudaMemcpyDeviceToDevice, s));
    } else {
        CTR_CUDA(cudaMemsetAsync(p->u, 0, nn * sizeof(T), s));
        CTR_CUDA(cudaMemsetAsync(p->Ru, 0, nm * sizeof(T), s));
        CTR_CUDA(cudaMemsetAsync(p->v1b, 0, nm * sizeof(T), s));
        CTR_CUDA(cudaMemsetAsync(p->v2b, 0, 2 * nn * sizeof(T), s));
        if (q.nonneg) CTR_CUDA(cudaMemsetAsync(p->ubar_u, 0, nn * sizeof(T), s));
    }
    ctr_diag local{};
    if ((st = pdrq_loop<T>(p, alpha, iters, q, beta, c, diag ? &local : nullptr, s)) != CTR_OK) return st;
    if (state) {
        CTR_CUDA(cudaMemcpyAsync(state->u, p->u, nn * sizeof(T), cudaMemcpyDeviceToDevice, s));
        CTR_CUDA(cudaMemcpyAsync(state->Ru, p->Ru, nm * sizeof(T), cudaMemcpyDeviceToDevice, s));
        CTR_CUDA(cudaMemcpyAsync(state->v1b, p->v1b, nm * sizeof(T), cudaMemcpyDeviceToDevice, s));
        CTR_CUDA(cudaMemcpyAsync(state->v2b, p->v2b, 2 * nn * sizeof(T), cudaMemcpyDeviceToDevice, s));
        if (q.nonneg) CTR_CUDA(cudaMemcpyAsync(state->ub, p->ubar_u, nn * sizeof(T), cudaMemcpyDeviceToDevice, s));
    }
    if (u_out) CTR_CUDA(cudaMemcpyAsync(u_out, p->u, nn * sizeof(T), cudaMemcpyDeviceToDevice, s));
    if (diag) {
        *diag = local;
        diag->beta = beta;
        diag->c = c;
    }
    return CTR_OK;
}

template <typename T>
ctr_status cp_impl(ctr_plan *p, const void *f, const uint8_t *mask, double alpha, double delta, int iters, double sp,
                   double sd, const ctr_params &q, void *u_out, ctr_diag *diag, void *stream)
{
    StreamJoin sj(p, stream);
    ctr_status st = sj.begin();
    if (st != CTR_OK) return st;
    cudaStream_t s = p->stream;
    double beta = q.beta;
    if (!(beta > 0)) {
        if ((st = power_beta<T>(p, q.power_iters, &beta, s)) != CTR_OK) return st;
        if (!(beta > 0)) return fail(CTR_ENUMERIC, "power iteration gave ||R_h|| = 0");
    }
    if ((st = build_desc_from_data<T>(p, (const T *)f, mask, delta, q.trace_ratio, beta, s)) != CTR_OK) return st;
    if (!(sp > 0) || !(sd > 0)) {
        // sigma tau (||Rt||^2 + 8/h^2) < 1 with ||Rt|| = 1 up to the power-iteration estimate
        const double step = 0.99 / std::sqrt(1.02 * (1.0 + 8.0 / (p->h * p->h)));
        sp = sd = step;
    }
    ctr_diag local{};
    if ((st = cp_loop<T>(p, alpha, iters, q, beta, sp, sd, diag ? &local : nullptr, s)) != CTR_OK) return st;
    CTR_CUDA(cudaMemcpyAsync(u_out, p->u, (size_t)p->n * p->n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    if (diag) {
        *diag = local;
        diag->beta = beta;
        diag->c = 0.0;
    }
    return CTR_OK;
}

}  // namespace
}  // namespace ctr

using namespace ctr;

extern "C" {

const char *ctr_last_error(void) { return g_last_error.c_str(); }

void ctr_default_params(ctr_params *q)
{
    if (!q) return;
    q->sigma = 1.0;
    q->tau = 1.0 / std::sqrt(8.0);
    q->eps = 0.0;          // resolved to pi/n
    q->c = 0.0;
    q->beta = 0.0;
    q->power_iters = 50;
    q->c_margin = 1.05;
    q->trace_ratio = 0.8;
    q->check_every = 0;
    q->stop_tol = 0.0;
    q->graph_block = 10;   // measured: 10 to 30 within 0.5 %, smaller graphs instantiate faster
    q->nonneg = 0;
    q->precond = 0;
}

size_t ctr_plan_device_bytes(const ctr_plan *p) { return p ? p->bytes : 0; }

ctr_status ctr_plan_history(ctr_plan *p, ctr_diag *out, int capacity, int *count)
{
    if (!p || !count) return fail(CTR_EINVAL, "plan and count must not be NULL");
    if (capacity < 0 || (capacity > 0 && !out)) return fail(CTR_EINVAL, "capacity must be >= 0 (out given when > 0)");
    DeviceGuard dg(p->device);
    if (!dg.ok) return fail(CTR_ECUDA, "cannot select the plan's device");
    *count = p->hist_count;
    const int k = capacity < p->hist_count ? capacity : p->hist_count;
    if (k <= 0) return CTR_OK;
    std::vector<double> h((size_t)k * HIST_FIELDS);
    CTR_CUDA(cudaMemcpyAsync(h.data(), p->d_hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    CTR_CUDA(cudaStreamSynchronize(p->stream));
    for (int r = 0; r < k; ++r) {
        const double *v = &h[(size_t)r * HIST_FIELDS];
        ctr_diag &d = out[r];
        d.beta = v[0];
        d.c = v[1];
        d.objective = v[2];
        d.data_fit = v[3];
        d.tv = v[4];
        d.violation = v[5];
        d.gap = v[6];
        d.dual_residual = v[7];
        d.rel_change = v[8];
        d.iters_done = (int)v[9];
    }
    return CTR_OK;
}

ctr_status ctr_plan_create(const ctr_geometry *g, ctr_dtype dtype, ctr_plan **out)
{
    if (!out) return fail(CTR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!g) return fail(CTR_EINVAL, "geometry is NULL");
    if (g->n < 1 || g->n_angles < 1 || g->n_bins < 1) return fail(CTR_EINVAL, "n, n_angles and n_bins must be >= 1");
    if (!(g->h > 0) || !(g->ds > 0) || !std::isfinite(g->h) || !std::isfinite(g->ds))
        return fail(CTR_EINVAL, "h and ds must be finite and > 0");
    if (!g->angles_host) return fail(CTR_EINVAL, "angles_host is NULL");
    if (g->n > 4096) return fail(CTR_EUNSUPPORTED, "n > 4096");
    if (g->n_angles > 65535) return fail(CTR_EUNSUPPORTED, "more than 65535 angles");
    if (g->ds / g->h > 2.5) return fail(CTR_EUNSUPPORTED, "ds/h > 2.5");
    if (dtype != CTR_F32 && dtype != CTR_F64 && dtype != CTR_BF16) return fail(CTR_EINVAL, "unknown dtype");
    for (int l = 0; l < g->n_angles; ++l)
        if (!std::isfinite(g->angles_host[l])) return fail(CTR_EINVAL, "non-finite angle");
    const double pmax = g->n_bins + 4.0 + 2.0 * g->n * (g->h / g->ds);
    ctr_plan *p = new (std::nothrow) ctr_plan();
    if (!p) return fail(CTR_ENOMEM, "host allocation failed");
    p->n = g->n;
    p->N = g->n_angles;
    p->M = g->n_bins;
    p->h = g->h;
    p->ds = g->ds;
    p->dtype = dtype;
    p->theta.assign(g->angles_host, g->angles_host + g->n_angles);
    if (dtype == CTR_F64) {
        int F = 62 - (int)std::ceil(std::log2(pmax));
        p->F = F > 48 ? 48 : F;
        p->esize = 8;
    } else {
        p->F = 32;
        p->esize = 4;
        p->bf16 = (dtype == CTR_BF16);
        if (pmax > (double)(1 << 28)) { destroy(p); return fail(CTR_EUNSUPPORTED, "geometry too large"); }
    }
    ctr_status st = fft_radices(p->n, p->radices);
    p->fft_ok = (st == CTR_OK);
    if (!p->fft_ok) p->radices.clear();
    st = CTR_OK;
    if (cudaGetDevice(&p->device) != cudaSuccess) { destroy(p); return fail(CTR_ECUDA, "no CUDA device"); }
    const size_t nn = (size_t)p->n * p->n, nm = (size_t)p->N * p->M, es = p->esize;
    p->red_blocks = 1024;
#define ALLOC(ptr, bytes)                                          \
    do {                                                           \
        void *tmp_ = nullptr;                                      \
        if ((st = alloc(p, &tmp_, (bytes))) != CTR_OK) {           \
            destroy(p);                                            \
            return st;                                             \
        }                                                          \
        ptr = (decltype(ptr))tmp_;                                 \
    } while (0)
    ALLOC(p->d_geom, sizeof(AngleGeom) * p->N);
    ALLOC(p->d_march, sizeof(AngleMarch) * p->N);
    ALLOC(p->d_twiddle, 2 * es * p->n);
    ALLOC(p->uT, es * nn);
    ALLOC(p->cbuf, 2 * es * nn);
    ALLOC(p->sym, es * nn);
    ALLOC(p->symh, es * nn);
    ALLOC(p->u, es * nn);
    ALLOC(p->du, es * nn);
    ALLOC(p->x, es * nn);
    ALLOC(p->xt, es * nn);
    ALLOC(p->y2, 2 * es * nn);
    ALLOC(p->v2b, 2 * es * nn);
    ALLOC(p->t2, 2 * es * nn);
    ALLOC(p->y1, es * nm);
    ALLOC(p->Ru, es * nm);
    ALLOC(p->v1b, es * nm);
    ALLOC(p->t1, es * nm);
    ALLOC(p->ubar_u, es * nn);
    ALLOC(p->pk_s, es * nn);
    ALLOC(p->aux, es * nn);
    p->ramp_L = ramp_length(p->M);
    if ((st = fft_radices(p->ramp_L, p->ramp_radices)) != CTR_OK) {
        destroy(p);
        return st;
    }
    ALLOC(p->d_ramp_tw, 2 * es * p->ramp_L);
    ALLOC(p->d_ramp_H, es * p->ramp_L);
    ALLOC(p->gs, es * nm);
    ALLOC(p->desc, 4 * es * nm);
    if (p->bf16) {
        ALLOC(p->uh, sizeof(__nv_bfloat16) * nn);
        ALLOC(p->uTh, sizeof(__nv_bfloat16) * nn);
        ALLOC(p->y1h, sizeof(__nv_bfloat16) * nm);
    }
    {
        // split the backprojection's angles into groups so that tiles x groups fills
        // the GPU (~8 CTAs of 4 warps per SM on 152 SMs); partial images are summed
        const int tiles = ((p->n + 31) / 32) * ((p->n + 31) / 32);
        int G = (1216 + tiles - 1) / tiles;
        if (G > MAX_BP_GROUPS) G = MAX_BP_GROUPS;
        const int maxg = p->N / 32 > 1 ? p->N / 32 : 1;
        if (G > maxg) G = maxg;
        p->bp_groups = G < 1 ? 1 : G;
        // room for up to MAX_BP_GROUPS groups at n <= 1024 so a tuner can change the split later
        int cap = p->bp_groups;
        if (p->n <= 1024) cap = maxg < MAX_BP_GROUPS ? (maxg > cap ? maxg : cap) : MAX_BP_GROUPS;
        p->bp_cap = cap;
        if (cap > 1) ALLOC(p->bp_part, es * nn * cap);
    }
    ALLOC(p->d_red, sizeof(double) * 8 * p->red_blocks);
    ALLOC(p->d_scal, sizeof(double) * 64);
    ALLOC(p->d_hist, sizeof(double) * HIST_FIELDS * MAX_CHECKS);
#undef ALLOC
    if ((st = build_tables(p)) != CTR_OK) { destroy(p); return st; }
    st = (dtype == CTR_F64) ? build_twiddles<double>(p) : build_twiddles<float>(p);
    if (st != CTR_OK) { destroy(p); return st; }
    st = (dtype == CTR_F64) ? configure_radon<double>(p) : configure_radon<float>(p);
    if (st == CTR_OK) st = (dtype == CTR_F64) ? configure_fft<double>(p) : configure_fft<float>(p);
    if (st != CTR_OK) { destroy(p); return st; }
    if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        destroy(p);
        return fail(CTR_ECUDA, "stream/event creation failed");
    }
    *out = p;
    return CTR_OK;
}

void ctr_plan_destroy(ctr_plan *p)
{
    if (!p) return;
    DeviceGuard dg(p->device);
    cudaDeviceSynchronize();
    destroy(p);
}

#define CTR_DISPATCH(p, call_f32, call_f64) ((p)->dtype == CTR_F64 ? (call_f64) : (call_f32))
#define CTR_GUARD(p)                                                                  \
    if (!(p)) return fail(CTR_EINVAL, "plan is NULL");                                \
    DeviceGuard dg_((p)->device);                                                     \
    if (!dg_.ok) return fail(CTR_ECUDA, "cannot select the plan's device");

ctr_status rh_forward(ctr_plan *p, const void *u, void *g, void *stream)
{
    CTR_NVTX("rh_forward");
    CTR_GUARD(p);
    if (!u || !g) return fail(CTR_EINVAL, "null buffer");
    cudaStream_t s = (cudaStream_t)stream;
    ctr_status st;
    if (p->dtype == CTR_F64) {
        if ((st = launch_transpose<double>(p, (const double *)u, (double *)p->uT, s)) != CTR_OK) return st;
        return op_forward<double>(p, (const double *)u, (const double *)p->uT, (double *)g, 1.0, s);
    }
    if (p->bf16) {
        if (fwd_needs_transpose<float>(p) &&
            (st = launch_transpose<__nv_bfloat16>(p, (const __nv_bfloat16 *)u, p->uTh, s)) != CTR_OK)
            return st;
        return op_forward_bf16(p, (const __nv_bfloat16 *)u, p->uTh, (float *)g, s);
    }
    if (fwd_needs_transpose<float>(p) && (st = launch_transpose<float>(p, (const float *)u, (float *)p->uT, s)) != CTR_OK)
        return st;
    return op_forward<float>(p, (const float *)u, (const float *)p->uT, (float *)g, 1.0, s);
}

ctr_status ctr_metal_trace(ctr_plan *p, const void *u, double threshold, int radius, double proj_tol,
                           uint8_t *marked, uint8_t *trace, void *stream)
{
    CTR_NVTX("ctr_metal_trace");
    CTR_GUARD(p);
    if (!u || !trace) return fail(CTR_EINVAL, "u and trace must not be NULL");
    if (!std::isfinite(threshold)) return fail(CTR_EINVAL, "threshold must be finite");
    if (radius < 0 || radius > 64) return fail(CTR_EINVAL, "radius must be in [0, 64]");
    if (!(proj_tol >= 0) || !std::isfinite(proj_tol)) return fail(CTR_EINVAL, "proj_tol must be finite and >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    return CTR_DISPATCH(p, metal_trace<float>(p, (const float *)u, threshold, radius, proj_tol, marked, trace, s),
                        metal_trace<double>(p, (const double *)u, threshold, radius, proj_tol, marked, trace, s));
}

ctr_status ctr_ramp_filter(ctr_plan *p, const void *g, void *y, void *stream)
{
    CTR_NVTX("ctr_ramp_filter");
    CTR_GUARD(p);
    if (!g || !y) return fail(CTR_EINVAL, "null buffer");
    cudaStream_t s = (cudaStream_t)stream;
    return CTR_DISPATCH(p, launch_ramp<float>(p, (const float *)g, (float *)y, nullptr, 1.0, s),
                        launch_ramp<double>(p, (const double *)g, (double *)y, nullptr, 1.0, s));
}

ctr_status ctr_fbp(ctr_plan *p, const void *g, void *u, void *stream)
{
    CTR_NVTX("ctr_fbp");
    CTR_GUARD(p);
    if (!g || !u) return fail(CTR_EINVAL, "null buffer");
    cudaStream_t s = (cudaStream_t)stream;
    const double w = 3.14159265358979323846 / p->N;   // the angle integral over [0, pi)
    ctr_status st;
    if (p->dtype == CTR_F64) {
        if ((st = launch_ramp<double>(p, (const double *)g, (double *)p->gs, nullptr, w, s)) != CTR_OK) return st;
        return op_adjoint<double>(p, (const double *)p->gs, (double *)u, 1.0, s);
    }
    if (p->bf16) {
        if ((st = launch_ramp<float>(p, (const float *)g, nullptr, p->y1h, w, s)) != CTR_OK) return st;
        return op_adjoint_bf16(p, p->y1h, (float *)u, s);
    }
    if ((st = launch_ramp<float>(p, (const float *)g, (float *)p->gs, nullptr, w, s)) != CTR_OK) return st;
    return op_adjoint<float>(p, (const float *)p->gs, (float *)u, 1.0, s);
}

ctr_status rh_forward_t(ctr_plan *p, const void *u, const void *uT, void *g, void *stream)
{
    CTR_NVTX("rh_forward_t");
    CTR_GUARD(p);
    if (!u || !uT || !g) return fail(CTR_EINVAL, "null buffer");
    cudaStream_t s = (cudaStream_t)stream;
    if (p->bf16) return op_forward_bf16(p, (const __nv_bfloat16 *)u, (const __nv_bfloat16 *)uT, (float *)g, s);
    return CTR_DISPATCH(p, op_forward<float>(p, (const float *)u, (const float *)uT, (float *)g, 1.0, s),
                        op_forward<double>(p, (const double *)u, (const double *)uT, (double *)g, 1.0, s));
}

unsigned long long ctr_plan_launch_count(const ctr_plan *p) { return p ? p->launches : 0ull; }
int ctr_plan_symmetric_jobs(const ctr_plan *p) { return p && p->orbit ? p->n_jobs : 0; }

ctr_status rh_adjoint(ctr_plan *p, const void *g, void *u, void *stream)
{
    CTR_NVTX("rh_adjoint");
    CTR_GUARD(p);
    if (!u || !g) return fail(CTR_EINVAL, "null buffer");
    cudaStream_t s = (cudaStream_t)stream;
    if (p->bf16) return op_adjoint_bf16(p, (const __nv_bfloat16 *)g, (float *)u, s);
    return CTR_DISPATCH(p, op_adjoint<float>(p, (const float *)g, (float *)u, 1.0, s),
                        op_adjoint<double>(p, (const double *)g, (double *)u, 1.0, s));
}

ctr_status precond_apply(ctr_plan *p, const ctr_params *prm, const void *y, void *x, void *stream)
{
    CTR_NVTX("precond_apply");
    CTR_GUARD(p);
    if (!prm || !y || !x) return fail(CTR_EINVAL, "null argument");
    ctr_params q = resolve(p, prm);
    ctr_status st = check_params(q);
    if (st != CTR_OK) return st;
    if (!(q.c > 0)) return fail(CTR_EINVAL, "precond_apply needs c > 0");
    if (!p->fft_ok) return fail(CTR_EUNSUPPORTED, "image size n must be of the form 2^a 3^b for the Fourier preconditioner");
    cudaStream_t s = (cudaStream_t)stream;
    if (p->dtype == CTR_F64) {
        if ((st = select_precond<double>(p, q, s)) != CTR_OK) return st;
        if ((st = launch_symbols<double>(p, q.sigma, q.tau, q.c, q.eps, s, q.nonneg != 0)) != CTR_OK) return st;
        return launch_circulant<double>(p, (const double *)y, false, (const double *)p->sym, (double *)x, 0, nullptr, nullptr, s);
    }
    if ((st = select_precond<float>(p, q, s)) != CTR_OK) return st;
    if ((st = launch_symbols<float>(p, q.sigma, q.tau, q.c, q.eps, s, q.nonneg != 0)) != CTR_OK) return st;
    return launch_circulant<float>(p, (const float *)y, false, (const float *)p->sym, (float *)x, 0, nullptr, nullptr, s);
}

static ctr_status validate_solve(ctr_plan *p, double alpha, int iters, const ctr_params &q)
{
    if (!p->fft_ok) return fail(CTR_EUNSUPPORTED, "image size n must be of the form 2^a 3^b for the Fourier preconditioner");
    if (!(alpha >= 0) || !std::isfinite(alpha)) return fail(CTR_EINVAL, "alpha must be finite and >= 0");
    if (iters < 0) return fail(CTR_EINVAL, "iters must be >= 0");
    if (q.check_every > 0 && iters / q.check_every > MAX_CHECKS)
        return fail(CTR_EINVAL, "iters / check_every exceeds the " + std::to_string(MAX_CHECKS) +
                                    " diagnostics records a plan holds");
    (void)p;
    return check_params(q);
}

ctr_status tv_cp_solve(ctr_plan *p, const void *f, const uint8_t *mask, double alpha, double delta, int iters,
                       double sigma_p, double tau_d, const ctr_params *prm, void *u_out, ctr_diag *diag,
                       void *stream)
{
    CTR_NVTX("tv_cp_solve");
    CTR_GUARD(p);
    if (!f || !u_out) return fail(CTR_EINVAL, "f and u_out must not be NULL");
    if (std::isnan(delta) || std::isnan(sigma_p) || std::isnan(tau_d)) return fail(CTR_EINVAL, "NaN argument");
    if (p->bf16) return fail(CTR_EUNSUPPORTED, "Alg. 1 runs on FP32 and FP64 plans");
    ctr_params q = resolve(p, prm);
    // no preconditioner: any n (validate_solve's FFT-size rule does not apply)
    if (!(alpha >= 0) || !std::isfinite(alpha)) return fail(CTR_EINVAL, "alpha must be finite and >= 0");
    if (iters < 0) return fail(CTR_EINVAL, "iters must be >= 0");
    ctr_status st = check_params(q);
    if (st != CTR_OK) return st;
    if (q.check_every > 0) return fail(CTR_EUNSUPPORTED, "check_every is implemented for Alg. 4, 5 and 3 solves");
    return CTR_DISPATCH(p, cp_impl<float>(p, f, mask, alpha, delta, iters, sigma_p, tau_d, q, u_out, diag, stream),
                        cp_impl<double>(p, f, mask, alpha, delta, iters, sigma_p, tau_d, q, u_out, diag, stream));
}

ctr_status tv_pd_solve(ctr_plan *p, const void *f, const uint8_t *mask, double alpha, double delta, int iters,
                       const ctr_params *prm, void *u_out, ctr_diag *diag, void *stream)
{
    CTR_NVTX("tv_pd_solve");
    CTR_GUARD(p);
    if (!f || !u_out) return fail(CTR_EINVAL, "f and u_out must not be NULL");
    if (std::isnan(delta)) return fail(CTR_EINVAL, "delta is NaN");
    ctr_params q = resolve(p, prm);
    ctr_status st = validate_solve(p, alpha, iters, q);
    if (st != CTR_OK) return st;
    return CTR_DISPATCH(p,
                        solve_impl<float>(p, f, mask, nullptr, nullptr, nullptr, nullptr, alpha, delta, iters, q, nullptr, u_out, diag, stream),
                        solve_impl<double>(p, f, mask, nullptr, nullptr, nullptr, nullptr, alpha, delta, iters, q, nullptr, u_out, diag, stream));
}

ctr_status tv_pdrq2_solve(ctr_plan *p, const void *f, double alpha, int iters, const ctr_params *prm, void *u_out,
                          ctr_diag *diag, void *stream)
{
    CTR_NVTX("tv_pdrq2_solve");
    CTR_GUARD(p);
    if (!f || !u_out) return fail(CTR_EINVAL, "f and u_out must not be NULL");
    ctr_params q = resolve(p, prm);
    ctr_status st = validate_solve(p, alpha, iters, q);
    if (st != CTR_OK) return st;
    if (q.nonneg) return fail(CTR_EUNSUPPORTED, "Alg. 3 has no non-negativity variant (nonneg = 0)");
    struct Alg3Scope {
        ctr_plan *p;
        explicit Alg3Scope(ctr_plan *pp) : p(pp) { p->alg3 = true; }
        ~Alg3Scope() { p->alg3 = false; }
    } scope(p);
    // (U_h): no metal trace, no data tolerance
    return CTR_DISPATCH(p,
                        solve_impl<float>(p, f, nullptr, nullptr, nullptr, nullptr, nullptr, alpha, -1.0, iters, q, nullptr, u_out, diag, stream),
                        solve_impl<double>(p, f, nullptr, nullptr, nullptr, nullptr, nullptr, alpha, -1.0, iters, q, nullptr, u_out, diag, stream));
}

ctr_status tv_admm_solve(ctr_plan *p, const void *f, double alpha, int iters, double mu, int cg_iters,
                         const ctr_params *prm, void *u_out, ctr_diag *diag, void *stream)
{
    CTR_NVTX("tv_admm_solve");
    CTR_GUARD(p);
    if (!f || !u_out) return fail(CTR_EINVAL, "f and u_out must not be NULL");
    if (!(mu > 0) || !std::isfinite(mu)) return fail(CTR_EINVAL, "mu must be finite and > 0");
    if (cg_iters < 1 || cg_iters > 64) return fail(CTR_EINVAL, "cg_iters must be in [1, 64]");
    if (p->bf16) return fail(CTR_EUNSUPPORTED, "ADMM runs on FP32 and FP64 plans");
    ctr_params q = resolve(p, prm);
    ctr_status st = validate_solve(p, alpha, iters, q);
    if (st != CTR_OK) return st;
    if (q.nonneg) return fail(CTR_EUNSUPPORTED, "ADMM solves the unconstrained problem (nonneg = 0)");
    if (q.check_every > 0) return fail(CTR_EUNSUPPORTED, "check_every is implemented for Alg. 4, 5 and 3 solves");
    auto run = [&](auto tag) -> ctr_status {
        using T = decltype(tag);
        StreamJoin sj(p, stream);
        ctr_status s2 = sj.begin();
        if (s2 != CTR_OK) return s2;
        cudaStream_t s = p->stream;
        if ((s2 = select_precond<T>(p, q, s)) != CTR_OK) return s2;
        double beta = q.beta;
        if (!(beta > 0)) {
            if ((s2 = power_beta<T>(p, q.power_iters, &beta, s)) != CTR_OK) return s2;
            if (!(beta > 0)) return fail(CTR_ENUMERIC, "power iteration gave ||R_h|| = 0");
        }
        double c = q.c;
        if (!(c > 0)) {
            double lam = 0;
            if ((s2 = power_lambda<T>(p, beta, q.eps, q.power_iters, &lam, s)) != CTR_OK) return s2;
            c = q.c_margin * lam;
            if (!(c > 0)) return fail(CTR_ENUMERIC, "power iteration gave c <= 0");
        }
        if ((s2 = build_desc_from_data<T>(p, (const T *)f, nullptr, -1.0, q.trace_ratio, beta, s)) != CTR_OK) return s2;
        ctr_diag local{};
        if ((s2 = admm_loop<T>(p, alpha, iters, cg_iters, mu, q, beta, c, diag ? &local : nullptr, s)) != CTR_OK)
            return s2;
        CTR_CUDA(cudaMemcpyAsync(u_out, p->u, (size_t)p->n * p->n * sizeof(T), cudaMemcpyDeviceToDevice, s));
        if (diag) {
            *diag = local;
            diag->beta = beta;
            diag->c = c;
        }
        return CTR_OK;
    };
    return p->dtype == CTR_F64 ? run(double{}) : run(float{});
}

ctr_status tv_mar_solve(ctr_plan *p, const void *f, double alpha, double delta, double threshold, int radius,
                        double proj_tol, int iters_pre, int iters, const ctr_params *prm, uint8_t *trace_out,
                        void *u_out, ctr_diag *diag, void *stream)
{
    CTR_NVTX("tv_mar_solve");
    CTR_GUARD(p);
    if (!f || !u_out || !trace_out) return fail(CTR_EINVAL, "f, trace_out and u_out must not be NULL");
    if (iters_pre < 1) return fail(CTR_EINVAL, "iters_pre must be >= 1");
    ctr_params q = resolve(p, prm);
    ctr_params q3 = q;
    q3.nonneg = 0;
    ctr_diag d3{};
    ctr_status st = tv_pdrq2_solve(p, f, alpha, iters_pre, &q3, u_out, &d3, stream);
    if (st != CTR_OK) return st;
    if ((st = ctr_metal_trace(p, u_out, threshold, radius, proj_tol, nullptr, trace_out, stream)) != CTR_OK) return st;
    q.beta = d3.beta;   // the same operator norm and constant c serve the second stage
    q.c = d3.c;
    return tv_pd_solve(p, f, trace_out, alpha, delta, iters, &q, u_out, diag, stream);
}

ctr_status tv_pd_run(ctr_plan *p, const void *w, const void *a, const void *lo, const void *hi, double alpha, int iters,
                     const ctr_params *prm, ctr_state *state, void *u_out, ctr_diag *diag, void *stream)
{
    CTR_NVTX("tv_pd_run");
    CTR_GUARD(p);
    if (!w || !a || !lo || !hi) return fail(CTR_EINVAL, "data-term arrays must not be NULL");
    if (!state && !u_out) return fail(CTR_EINVAL, "state and u_out are both NULL");
    if (state && (!state->u || !state->Ru || !state->v1b || !state->v2b)) return fail(CTR_EINVAL, "state has a NULL buffer");
    ctr_params q = resolve(p, prm);
    if (state && q.nonneg && !state->ub) return fail(CTR_EINVAL, "nonneg: state->ub (bar u) must be given");
    ctr_status st = validate_solve(p, alpha, iters, q);
    if (st != CTR_OK) return st;
    return CTR_DISPATCH(p,
                        solve_impl<float>(p, nullptr, nullptr, w, a, lo, hi, alpha, 0.0, iters, q, state, u_out, diag, stream),
                        solve_impl<double>(p, nullptr, nullptr, w, a, lo, hi, alpha, 0.0, iters, q, state, u_out, diag, stream));
}

ctr_status tv_pd_solve_state(ctr_plan *p, const void *f, const uint8_t *mask, double alpha, double delta, int iters,
                             const ctr_params *prm, ctr_state *state, ctr_diag *diag, void *stream)
{
    CTR_NVTX("tv_pd_solve_state");
    CTR_GUARD(p);
    if (!f || !state || !state->u || !state->Ru || !state->v1b || !state->v2b)
        return fail(CTR_EINVAL, "f and every state buffer must be given");
    if (std::isnan(delta)) return fail(CTR_EINVAL, "delta is NaN");
    if (p->bf16) return fail(CTR_EUNSUPPORTED, "state-carrying solves need an FP32 or FP64 plan");
    ctr_params q = resolve(p, prm);
    if (q.nonneg && !state->ub) return fail(CTR_EINVAL, "nonneg: state->ub (bar u) must be given");
    ctr_status st = validate_solve(p, alpha, iters, q);
    if (st != CTR_OK) return st;
    return CTR_DISPATCH(p,
                        solve_impl<float>(p, f, mask, nullptr, nullptr, nullptr, nullptr, alpha, delta, iters, q, state, nullptr, diag, stream),
                        solve_impl<double>(p, f, mask, nullptr, nullptr, nullptr, nullptr, alpha, delta, iters, q, state, nullptr, diag, stream));
}

ctr_status tv_pd_vjp_step(ctr_plan *p, const void *f, const uint8_t *mask, double alpha, double delta,
                          const ctr_params *prm, const ctr_state *s0, const ctr_state *s1, void *bu, void *b1,
                          void *b2, void *gf, double *galpha_dev, void *stream)
{
    CTR_NVTX("tv_pd_vjp_step");
    CTR_GUARD(p);
    if (!f || !s0 || !s1 || !bu || !b1 || !b2 || !gf || !galpha_dev) return fail(CTR_EINVAL, "null argument");
    if (!s0->u || !s0->v1b || !s0->v2b || !s1->u || !s1->Ru) return fail(CTR_EINVAL, "state buffer missing");
    if (p->bf16) return fail(CTR_EUNSUPPORTED, "the reverse mode needs an FP32 or FP64 plan");
    ctr_params q = resolve(p, prm);
    if (q.nonneg) return fail(CTR_EUNSUPPORTED, "the reverse mode covers Alg. 4 only (nonneg = 0)");
    ctr_status st = validate_solve(p, alpha, 1, q);
    if (st != CTR_OK) return st;
    if (!(q.beta > 0) || !(q.c > 0)) return fail(CTR_EINVAL, "the reverse mode needs beta and c given (> 0)");
    cudaStream_t s = (cudaStream_t)stream;
    st = p->dtype == CTR_F64 ? select_precond<double>(p, q, s) : select_precond<float>(p, q, s);
    if (st != CTR_OK) return st;
    if (p->dtype == CTR_F64)
        return pdrq_vjp_step<double>(p, (const double *)s0->u, (const double *)s0->v1b, (const double *)s0->v2b,
                                     (const double *)s1->u, (const double *)s1->Ru, (const double *)f, mask, delta,
                                     q.trace_ratio, alpha, q.beta, q.c, q, (double *)bu, (double *)b1, (double *)b2,
                                     (double *)gf, galpha_dev, s);
    return pdrq_vjp_step<float>(p, (const float *)s0->u, (const float *)s0->v1b, (const float *)s0->v2b,
                                (const float *)s1->u, (const float *)s1->Ru, (const float *)f, mask, delta,
                                q.trace_ratio, alpha, q.beta, q.c, q, (float *)bu, (float *)b1, (float *)b2,
                                (float *)gf, galpha_dev, s);
}

ctr_status tv_pd_vjp_segment(ctr_plan *p, const void *f, const uint8_t *mask, double alpha, double delta,
                             const ctr_params *prm, const ctr_state *s_start, int length, void *workspace, void *bu,
                             void *b1, void *b2, void *gf, double *galpha_dev, void *stream)
{
    CTR_NVTX("tv_pd_vjp_segment");
    CTR_GUARD(p);
    if (!f || !s_start || !workspace || !bu || !b1 || !b2 || !gf || !galpha_dev) return fail(CTR_EINVAL, "null argument");
    if (!s_start->u || !s_start->Ru || !s_start->v1b || !s_start->v2b) return fail(CTR_EINVAL, "state buffer missing");
    if (length < 1) return fail(CTR_EINVAL, "length must be >= 1");
    if (p->bf16) return fail(CTR_EUNSUPPORTED, "the reverse mode needs an FP32 or FP64 plan");
    ctr_params q = resolve(p, prm);
    if (q.nonneg) return fail(CTR_EUNSUPPORTED, "the reverse mode covers Alg. 4 only (nonneg = 0)");
    ctr_status st = validate_solve(p, alpha, 1, q);
    if (st != CTR_OK) return st;
    if (!(q.beta > 0) || !(q.c > 0)) return fail(CTR_EINVAL, "the reverse mode needs beta and c given (> 0)");
    q.check_every = 0;   // the replay keeps no diagnostics history
    q.stop_tol = 0.0;
    auto run = [&](auto tag) -> ctr_status {
        using T = decltype(tag);
        cudaStream_t s = (cudaStream_t)stream;
        const size_t nn = (size_t)p->n * p->n, nm = (size_t)p->N * p->M, per = 3 * nn + 2 * nm;
        T *ws = (T *)workspace;
        auto slot = [&](int k, int part) -> T * {   // 0: u, 1: Ru, 2: v1b, 3: v2b
            T *b = ws + (size_t)k * per;
            return part == 0 ? b : part == 1 ? b + nn : part == 2 ? b + nn + nm : b + nn + 2 * nm;
        };
        ctr_status s2;
        if ((s2 = select_precond<T>(p, q, s)) != CTR_OK) return s2;
        if ((s2 = build_desc_from_data<T>(p, (const T *)f, mask, delta, q.trace_ratio, q.beta, s)) != CTR_OK) return s2;
        CTR_CUDA(cudaMemcpyAsync(p->u, s_start->u, nn * sizeof(T), cudaMemcpyDeviceToDevice, s));
        CTR_CUDA(cudaMemcpyAsync(p->Ru, s_start->Ru, nm * sizeof(T), cudaMemcpyDeviceToDevice, s));
        CTR_CUDA(cudaMemcpyAsync(p->v1b, s_start->v1b, nm * sizeof(T), cudaMemcpyDeviceToDevice, s));
        CTR_CUDA(cudaMemcpyAsync(p->v2b, s_start->v2b, 2 * nn * sizeof(T), cudaMemcpyDeviceToDevice, s));
        auto save = [&](int k) -> ctr_status {
            CTR_CUDA(cudaMemcpyAsync(slot(k, 0), p->u, nn * sizeof(T), cudaMemcpyDeviceToDevice, s));
            CTR_CUDA(cudaMemcpyAsync(slot(k, 1), p->Ru, nm * sizeof(T), cudaMemcpyDeviceToDevice, s));
            CTR_CUDA(cudaMemcpyAsync(slot(k, 2), p->v1b, nm * sizeof(T), cudaMemcpyDeviceToDevice, s));
            CTR_CUDA(cudaMemcpyAsync(slot(k, 3), p->v2b, 2 * nn * sizeof(T), cudaMemcpyDeviceToDevice, s));
            return CTR_OK;
        };
        if ((s2 = save(0)) != CTR_OK) return s2;
        for (int k = 0; k < length; ++k) {           // replay, keeping every state
            if ((s2 = pdrq_loop<T>(p, alpha, 1, q, q.beta, q.c, nullptr, s)) != CTR_OK) return s2;
            if ((s2 = save(k + 1)) != CTR_OK) return s2;
        }
        for (int k = length - 1; k >= 0; --k)        // and reverse it, newest first
            if ((s2 = pdrq_vjp_step<T>(p, slot(k, 0), slot(k, 2), slot(k, 3), slot(k + 1, 0), slot(k + 1, 1),
                                       (const T *)f, mask, delta, q.trace_ratio, alpha, q.beta, q.c, q, (T *)bu,
                                       (T *)b1, (T *)b2, (T *)gf, galpha_dev, s)) != CTR_OK)
                return s2;
        return CTR_OK;
    };
    return p->dtype == CTR_F64 ? run(double{}) : run(float{});
}

ctr_status ctr_plan_set_fwd_shape(ctr_plan *p, int jobs_per_cta, int segments)
{
    if (!p) return fail(CTR_EINVAL, "plan is NULL");
    const int key = jobs_per_cta * 16 + segments;
    if (key != 1 * 16 + 2 && key != 1 * 16 + 4 && key != 1 * 16 + 8 && key != 2 * 16 + 2 && key != 2 * 16 + 4 &&
        key != 4 * 16 + 2 && key != 4 * 16 + 1)
        return fail(CTR_EINVAL, "forward shape must be (1, 2), (1, 4), (1, 8), (2, 2), (2, 4), (4, 2) or (4, 1)");
    if (!p->orbit) return fail(CTR_EUNSUPPORTED, "the plan projects angle by angle (no symmetric forward projector)");
    if (key == 4 * 16 + 1 && p->stg_wmax <= 0)
        return fail(CTR_EUNSUPPORTED, "the staged forward shape (4, 1): its orbit-image window exceeds shared memory "
                                      "on this geometry");
    p->fwd_slots = jobs_per_cta;
    p->fwd_segs = segments;
    return CTR_OK;
}

ctr_status ctr_plan_set_fft_form(ctr_plan *p, int form)
{
    if (!p) return fail(CTR_EINVAL, "plan is NULL");
    if (form != 0 && form != 1) return fail(CTR_EINVAL, "fft form must be 0 (warp-level) or 1 (CTA-level)");
    p->fft_form = form;
    return CTR_OK;
}

ctr_status ctr_plan_set_launch_overlap(ctr_plan *p, int on)
{
    if (!p) return fail(CTR_EINVAL, "plan is NULL");
    if (on != 0 && on != 1) return fail(CTR_EINVAL, "launch overlap must be 0 or 1");
    p->pdl = on;
    return CTR_OK;
}

int ctr_plan_get_launch_overlap(const ctr_plan *p) { return p ? p->pdl : -1; }

int ctr_plan_get_fft_form(const ctr_plan *p)
{
    if (!p) return -1;
    return (p->fft_form == 0 && wfft_supported(p)) ? 0 : 1;
}

ctr_status ctr_plan_get_fwd_shape(const ctr_plan *p, int *jobs_per_cta, int *segments)
{
    if (!p || !jobs_per_cta || !segments) return fail(CTR_EINVAL, "null argument");
    *jobs_per_cta = p->orbit ? p->fwd_slots : 0;
    *segments = p->orbit ? p->fwd_segs : 0;
    return CTR_OK;
}

ctr_status ctr_plan_set_bp_groups(ctr_plan *p, int groups)
{
    if (!p) return fail(CTR_EINVAL, "plan is NULL");
    if (p->orbit) {
        if (groups < 1 || groups > p->obp_cap)
            return fail(CTR_EINVAL, "groups must be in [1, " + std::to_string(p->obp_cap) + "]");
        p->obp_groups = groups;
        return CTR_OK;
    }
    if (groups < 1 || groups > p->bp_cap || groups > p->N)
        return fail(CTR_EINVAL, "groups must be in [1, " + std::to_string(p->bp_cap < p->N ? p->bp_cap : p->N) + "]");
    p->bp_groups = groups;
    return CTR_OK;
}

int ctr_plan_get_bp_groups(const ctr_plan *p) { return p ? (p->orbit ? p->obp_groups : p->bp_groups) : 0; }

void ctr_batch_destroy(ctr_batch *b)
{
    if (!b) return;
    DeviceGuard dg(b->device);
    cudaDeviceSynchronize();
    for (ctr_plan *p : b->plans) ctr_plan_destroy(p);
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_prefix) cudaFree(b->d_prefix);
    if (b->d_gb) cudaFree(b->d_gb);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    delete b;
}

ctr_status ctr_batch_create(const ctr_geometry *geos, int count, ctr_batch **out)
{
    if (!out || !geos || count < 1) return fail(CTR_EINVAL, "geos/out NULL or count < 1");
    *out = nullptr;
    ctr_batch *b = new (std::nothrow) ctr_batch();
    if (!b) return fail(CTR_ENOMEM, "host allocation failed");
    if (cudaGetDevice(&b->device) != cudaSuccess) { delete b; return fail(CTR_ECUDA, "no CUDA device"); }
    ctr_status st = CTR_OK;
    for (int i = 0; i < count && st == CTR_OK; ++i) {
        ctr_plan *p = nullptr;
        st = ctr_plan_create(&geos[i], CTR_F32, &p);
        if (st != CTR_OK) break;
        b->plans.push_back(p);
        if (!p->fft_ok) st = fail(CTR_EUNSUPPORTED, "slice " + std::to_string(i) + ": n must be 2^a 3^b");
        else if (p->ncand != 2 || p->h > p->ds)
            st = fail(CTR_EUNSUPPORTED, "slice " + std::to_string(i) + ": batched solve needs ds/h in [1, sqrt(2))");
    }
    if (st == CTR_OK) {
        if (cudaMalloc((void **)&b->d_desc, sizeof(SliceDesc) * count) != cudaSuccess ||
            cudaMalloc((void **)&b->d_prefix, sizeof(int) * BS_COUNT * (count + 1)) != cudaSuccess ||
            cudaMalloc((void **)&b->d_gb, sizeof(GridBarrier)) != cudaSuccess) {
            cudaGetLastError();
            st = fail(CTR_ENOMEM, "batch tables: cudaMalloc failed");
        }
    }
    if (st == CTR_OK && (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
                         cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess))
        st = fail(CTR_ECUDA, "stream/event creation failed");
    if (st == CTR_OK) st = batch_prepare(b);
    if (st != CTR_OK) {
        std::string msg = g_last_error;
        ctr_batch_destroy(b);
        return fail(st, msg);
    }
    *out = b;
    return CTR_OK;
}

ctr_status ctr_batch_retune(ctr_batch *b)
{
    if (!b) return fail(CTR_EINVAL, "batch is NULL");
    DeviceGuard dg(b->device);
    return batch_prepare(b);
}

ctr_plan *ctr_batch_plan(ctr_batch *b, int i)
{
    if (!b || i < 0 || i >= (int)b->plans.size()) return nullptr;
    return b->plans[i];
}

unsigned long long ctr_batch_launch_count(const ctr_batch *b) { return b ? b->launches : 0ull; }

ctr_status ctr_batch_set_mode(ctr_batch *b, int mode, unsigned long long spin_limit)
{
    if (!b) return fail(CTR_EINVAL, "batch is NULL");
    if (mode != 0 && mode != 1) return fail(CTR_EINVAL, "mode must be 0 or 1");
    if (mode == 1 && b->persist_grid <= 0)
        return fail(CTR_EUNSUPPORTED, "the persistent iteration does not fit on this device (shared memory or registers)");
    b->mode = mode;
    b->spin_limit = spin_limit;
    return CTR_OK;
}

int ctr_batch_get_mode(const ctr_batch *b) { return b ? b->mode : -1; }
int ctr_batch_persistent_ctas(const ctr_batch *b) { return b ? b->persist_grid : 0; }

ctr_status tv_pd_solve_batched(ctr_batch *b, const void *const *f_devs, const uint8_t *const *masks,
                               const double *alphas, const double *deltas, int iters, const ctr_params *prm,
                               const double *betas, const double *cs, void *const *u_outs, ctr_diag *diags,
                               void *stream)
{
    CTR_NVTX("tv_pd_solve_batched");
    if (!b) return fail(CTR_EINVAL, "batch is NULL");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail(CTR_ECUDA, "cannot select the batch's device");
    const int ns = (int)b->plans.size();
    if (!f_devs || !alphas || !deltas || !u_outs) return fail(CTR_EINVAL, "f_devs, alphas, deltas, u_outs must not be NULL");
    for (int i = 0; i < ns; ++i) {
        if (!f_devs[i] || !u_outs[i]) return fail(CTR_EINVAL, "slice " + std::to_string(i) + ": NULL buffer");
        if (!(alphas[i] >= 0) || !std::isfinite(alphas[i]) || std::isnan(deltas[i]))
            return fail(CTR_EINVAL, "slice " + std::to_string(i) + ": alpha must be finite >= 0, delta not NaN");
    }
    if (iters < 0) return fail(CTR_EINVAL, "iters must be >= 0");
    ctr_params q;
    ctr_default_params(&q);
    if (prm) q = *prm;
    ctr_params qc = q;
    if (!(qc.eps > 0)) qc.eps = 1.0;     // validated per slice (pi/n when unset)
    ctr_status st = check_params(qc);
    if (st != CTR_OK) return st;
    if (q.check_every > 0) return fail(CTR_EUNSUPPORTED, "check_every is implemented for single-plan solves");
    CTR_CUDA(cudaEventRecord(b->ev_in, (cudaStream_t)stream));
    CTR_CUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    st = batch_solve(b, (const float *const *)f_devs, masks, alphas, deltas, iters, q, betas, cs,
                     (float *const *)u_outs, diags, b->stream);
    cudaEventRecord(b->ev_out, b->stream);
    cudaStreamWaitEvent((cudaStream_t)stream, b->ev_out, 0);
    return st;
}

ctr_status ctr_power_beta(ctr_plan *p, int iters, double *beta_out, void *stream)
{
    CTR_NVTX("ctr_power_beta");
    CTR_GUARD(p);
    if (!beta_out || iters < 1) return fail(CTR_EINVAL, "beta_out NULL or iters < 1");
    StreamJoin sj(p, stream);
    ctr_status st = sj.begin();
    if (st != CTR_OK) return st;
    return CTR_DISPATCH(p, power_beta<float>(p, iters, beta_out, p->stream), power_beta<double>(p, iters, beta_out, p->stream));
}

ctr_status ctr_power_lambda(ctr_plan *p, double beta, double eps, int iters, double *lam, void *stream)
{
    CTR_NVTX("ctr_power_lambda");
    CTR_GUARD(p);
    if (!lam || iters < 1 || !(beta > 0) || !(eps > 0)) return fail(CTR_EINVAL, "bad argument");
    if (!p->fft_ok) return fail(CTR_EUNSUPPORTED, "image size n must be of the form 2^a 3^b for the Fourier preconditioner");
    StreamJoin sj(p, stream);
    ctr_status st = sj.begin();
    if (st != CTR_OK) return st;
    p->precond_kind = 0;   // this entry point is the inverse-norm form; solves choose their own
    return CTR_DISPATCH(p, power_lambda<float>(p, beta, eps, iters, lam, p->stream),
                        power_lambda<double>(p, beta, eps, iters, lam, p->stream));
}

ctr_status ctr_grad(ctr_plan *p, const void *u, void *px, void *stream)
{
    CTR_GUARD(p);
    if (!u || !px) return fail(CTR_EINVAL, "null buffer");
    cudaStream_t s = (cudaStream_t)stream;
    return CTR_DISPATCH(p, op_grad<float>(p, (const float *)u, (float *)px, s), op_grad<double>(p, (const double *)u, (double *)px, s));
}

ctr_status ctr_div(ctr_plan *p, const void *px, void *d, void *stream)
{
    CTR_GUARD(p);
    if (!px || !d) return fail(CTR_EINVAL, "null buffer");
    cudaStream_t s = (cudaStream_t)stream;
    return CTR_DISPATCH(p, op_div<float>(p, (const float *)px, (float *)d, s), op_div<double>(p, (const double *)px, (double *)d, s));
}

}  // extern "C"
