// The projectors (radon.cu), the FFT passes (fft.cu) and the persistent batched
// iteration below form one translation unit, so that the persistent kernel can inline
// every stage body of Alg. 4 (they live in the two files' internal namespaces).
//
// Persistent batched iteration: one cooperative launch runs a whole iteration of Alg. 4
// for every slice of a batch.  The launch holds as many CTAs of 256 threads as can be
// resident at once; each phase of the iteration is a grid-stride loop over the virtual
// blocks of its stages (the same bodies, block maps and shared-memory layouts as the
// one-launch-per-stage form, so the results are identical), and the phases are separated
// by a grid barrier:
//   1  backprojection (per-angle and symmetric slices)      step A of Alg. 4
//   2  forward row FFTs (fold of the partial images)         step B
//   3  column FFTs with the symbol
//   4  inverse row FFTs (u += ...)
//   5  orbit images and the TV dual step                     steps C (input) and D
//   6  forward projection with the data-dual epilogue        step C
// Stage bodies written for 128-thread CTAs run on the first half of the CTA and
// synchronise with a named barrier; the second half waits at the block barrier after
// each body.  The grid barrier spins a bounded number of times; when the count runs out
// it sets the status word, every CTA leaves, and the host reports CTR_ETIMEOUT.
#include "radon.cu"
#include "fft.cu"

namespace ctr {
namespace {

constexpr int PERSIST_THREADS = 256;

// Sense by generation: the last CTA to arrive resets the count and bumps the
// generation; the others spin on the generation (at most spin_limit polls).  Returns
// false (in every thread of the CTA) once any CTA has given up.
__device__ __forceinline__ bool grid_barrier(GridBarrier *gb, unsigned nblocks, unsigned long long spin_limit)
{
    __shared__ int s_go;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &gb->gen;
        volatile int *vstat = &gb->status;
        const unsigned g = *vgen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(&gb->count, 1u) + 1u == nblocks) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            unsigned long long polls = 0;
            while (*vgen == g) {
                if (polls++ >= spin_limit || *vstat != 0) {
                    atomicOr(&gb->status, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_go = ok && *vstat == 0;
    }
    __syncthreads();
    return s_go != 0;
}

// One virtual block of stage `stg`.
__device__ __forceinline__ void persist_stage_block(int stg, const SliceDesc *__restrict__ sd,
                                                    const int *__restrict__ pre, int ns, int vb)
{
    const int tid = threadIdx.x;
    switch (stg) {
    case BS_BP: {
        if (tid >= 32 * BP_TY) return;
        const int s = find_slice(pre, ns, vb);
        const SliceDesc &d = sd[s];
        const int local = vb - pre[s];
        const int bx = local % d.bp_tiles_x, rest = local / d.bp_tiles_x;
        bp_body<float, float, true>(d.y1, d.n, d.N, d.M, 32, d.wstride, d.per_group, d.geom, d.bpe,
                                    d.bp_groups > 1 ? d.bp_part : nullptr, bx, rest % d.bp_tiles_y,
                                    rest / d.bp_tiles_y);
        return;
    }
    case BS_BP_SYM: {
        const int s = find_slice(pre, ns, vb);
        const SliceDesc &d = sd[s];
        const int local = vb - pre[s];
        const int bx = local % d.bp_tiles_x, rest = local / d.bp_tiles_x;
        obp_body<float>(d.y1, d.n, d.M, d.wstride, d.per_group, d.n_jobs, d.jobs, d.bp_part, bx,
                        rest % d.bp_tiles_y, rest / d.bp_tiles_y);
        return;
    }
    case BS_FFT_ROWS: {
        const int s = find_slice_fft(pre, ns, vb);
        const SliceDesc &d = sd[s];
        RowsInput<float> src{};
        if (d.orbit || d.bp_groups > 1) {
            src.part = d.bp_part;
            src.groups = d.bp_groups;
            src.orbit = d.orbit;
            src.epi = d.bpe;
        }
        if (d.packed) fft_rows_fwd_packed_body<float>(src, d.cbuf, d.n, d.prp, d.fp, d.tw, vb - pre[s]);
        else fft_rows_fwd_body<float>(src, d.cbuf, d.n, d.rpc, d.fp, d.tw, vb - pre[s]);
        return;
    }
    case BS_FFT_COLS: {
        const int s = find_slice_fft(pre, ns, vb);
        const SliceDesc &d = sd[s];
        if (d.packed) fft_cols_body<float>(d.cbuf, d.sym, d.n, d.pcw, d.fp, d.tw, vb - pre[s], 0, d.n / 2 + 1, d.n / 2 + 1);
        else fft_cols_body<float>(d.cbuf, d.sym, d.n, d.cw, d.fp, d.tw, vb - pre[s], d.twist);
        return;
    }
    case BS_FFT_ROWS_INV: {
        const int s = find_slice_fft(pre, ns, vb);
        const SliceDesc &d = sd[s];
        if (d.packed)
            fft_rows_inv_packed_body<float>(d.cbuf, d.n, d.prp, d.fp, d.tw, d.u, 1, d.orbit ? nullptr : d.uT, nullptr,
                                            nullptr, nullptr, vb - pre[s]);
        else
            fft_rows_inv_body<float>(d.cbuf, d.n, d.rpc, d.fp, d.tw, d.u, 1, d.orbit ? nullptr : d.uT, nullptr, nullptr,
                                     nullptr, vb - pre[s]);
        return;
    }
    case BS_ORBIT: {
        const int s = find_slice(pre, ns, vb);
        const SliceDesc &d = sd[s];
        const int local = vb - pre[s], tiles = (d.n + 31) / 32;
        orbit_image_body<float>(d.u, d.ubar, d.n, local % tiles, local / tiles);
        return;
    }
    case BS_TV: {
        const int s = find_slice(pre, ns, vb);
        const SliceDesc &d = sd[s];
        const TvDualJob<float> job{d.u, d.n, d.sigma, d.tau, d.lam, d.inv_h, d.v2b, d.y2, nullptr, d.ub};
        const size_t nn = (size_t)d.n * d.n, nb = (size_t)(pre[s + 1] - pre[s]);
        for (size_t e = (size_t)(vb - pre[s]) * blockDim.x + tid; e < nn; e += nb * blockDim.x)
            tv_dual_at(job, pix_i(e, d.n), pix_j(e, d.n));
        return;
    }
    case BS_FWD: {
        if (tid >= FWD_THREADS) return;
        const int s = find_slice(pre, ns, vb);
        const SliceDesc &d = sd[s];
        const int local = vb - pre[s];
        fwd_body<float, float, 2, true>(d.u, d.uT, d.n, d.N, d.M, 32, d.march, d.fwe, local % d.fwd_chunks,
                                        local / d.fwd_chunks);
        return;
    }
    case BS_FWD_SYM: {
        if (tid >= ORBIT_THREADS) return;
        const int s = find_slice(pre, ns, vb);
        const SliceDesc &d = sd[s];
        const int local = vb - pre[s];
        forward_orbit_body<float, true>(d.ubar, d.n, d.n_jobs, d.M, d.jobs, d.fwe, local % d.fwd_chunks,
                                        local / d.fwd_chunks);
        return;
    }
    default:
        return;
    }
}

__global__ void __launch_bounds__(PERSIST_THREADS, 1)
k_batch_iteration(const SliceDesc *__restrict__ sd, const int *__restrict__ prefix, int ns, GridBarrier *gb,
                  unsigned long long spin_limit)
{
    static_assert(32 * BP_TY <= PERSIST_THREADS && FWD_THREADS <= PERSIST_THREADS && ORBIT_THREADS <= PERSIST_THREADS &&
                      32 * OBP_TY == PERSIST_THREADS && FFT_THREADS == PERSIST_THREADS,
                  "stage bodies must fit the persistent CTA");
    constexpr int PHASES = 6;
    const int phase_stage[PHASES][2] = {{BS_BP, BS_BP_SYM}, {BS_FFT_ROWS, -1}, {BS_FFT_COLS, -1},
                                        {BS_FFT_ROWS_INV, -1}, {BS_ORBIT, BS_TV}, {BS_FWD, BS_FWD_SYM}};
    const int stride = ns + 1;
    for (int ph = 0; ph < PHASES; ++ph) {
        for (int q = 0; q < 2; ++q) {
            const int stg = phase_stage[ph][q];
            if (stg < 0) continue;
            const int *pre = prefix + stg * stride;
            const int total = pre[ns];
            for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
                persist_stage_block(stg, sd, pre, ns, vb);
                __syncthreads();                       // the body's shared memory is reused next
            }
        }
        if (ph + 1 < PHASES && !grid_barrier(gb, gridDim.x, spin_limit)) return;
    }
}

}  // namespace

// Resident CTAs per SM of the persistent kernel with `smem` bytes of dynamic shared
// memory (0 when it does not fit).
int persist_blocks_per_sm(size_t smem)
{
    if (raise_smem_limit(k_batch_iteration, smem) != CTR_OK) {
        (void)cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_iteration, PERSIST_THREADS, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return nb;
}

ctr_status launch_batch_iteration(const SliceDesc *sd, const int *prefix, int ns, GridBarrier *gb,
                                  unsigned long long spin_limit, int grid, size_t smem, cudaStream_t s)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(PERSIST_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CTR_CUDA(cudaLaunchKernelEx(&cfg, k_batch_iteration, sd, prefix, ns, gb, spin_limit));
    return CTR_OK;
}

}  // namespace ctr
