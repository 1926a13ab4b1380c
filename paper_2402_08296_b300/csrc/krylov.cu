// Fine operator, preconditioner application and the flexible CG driver.
//
// Preconditioner (Section III-A): restriction with |R_i r| and the coarse
// right-hand side R_0 r (Eq. 13's input), the coarse solve as a GEMV with the
// setup's explicit inverse of A_0, the local solves (DSS inference, Eq. 14, or
// band Cholesky, Eq. 7), and the gluing z = r_c + sum_i R_i^T |R_i r| r~_i
// (Eq. 16) as a node-centric gather over each node's sorted subdomain list,
// so every z_j is summed in a fixed order without atomics.
//
// Krylov: flexible CG with truncation m (Notay 2000): the new direction is
// A-orthogonalised against the last m ones, p_k = z_k - sum_j (z_k.q_j)/(p_j.q_j) p_j,
// alpha = (p_k.r_k)/(p_k.q_k).  With m = 1 and a fixed SPD preconditioner it
// generates the iterates of Algorithm 1.  All vectors and dot products are
// FP64; every reduction uses a fixed grid and a fixed summation tree, so a
// solve is bitwise reproducible.  Scalars stay on the device; the host only
// polls a stop flag every few iterations.
#include "ddg_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

namespace ddg {

constexpr int KT = 256;            // threads per block of the vector kernels
constexpr int RB = 1184;           // grid of the norm kernels; bound on the reducing kernels' grids (partials per sum)
constexpr int PUG = 592;           // grid of the direction update (4 CTAs of 256 per SM)
constexpr int MAXM = 16;           // largest truncation
constexpr int POLL = 4;            // iterations between stop-flag polls
constexpr int HIST_MAX = 1 << 20;  // iterations a solve's residual history keeps at most
constexpr int OFF_MD = 0;          // partial-sum regions of kpart: multidot, then SpMV dots, then |r|^2

// scalar slots (kscal) and flags (kflag)
enum { S_BNORM = 0, S_ALPHA = 1, S_REL = 2, S_R0 = 3, S_BETA = 8, S_PQ = 8 + MAXM, S_COUNT = 8 + 2 * MAXM };
enum { F_STOP = 0, F_ITERS = 1, F_T_MD = 2, F_T_SP = 3, F_T_XR = 4, F_COUNT = 5 };

// Block sums of NV per-thread values, written to out[j * stride] for j < nv.  This part runs
// FP64 at about 1/64 of its FP32 rate, so every FP64 instruction of a warp holds its
// sub-partition's FP64 pipe for about 64 cycles, and a shuffle tree in every warp for every
// sum (5 additions per warp and sum) costs more than the dot products themselves.  Instead
// the values go through shared memory and warp j sums column j: KT/32 - 1 + 5 additions per
// sum, in a fixed order.  sh holds nv * KT doubles.
template <int NV>
__device__ __forceinline__ void block_parts(const double (&v)[NV], int nv, double *sh, double *out, long long stride) {
#pragma unroll
    for (int j = 0; j < NV; ++j)
        if (j < nv) sh[j * KT + threadIdx.x] = v[j];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = warp; j < nv; j += KT / 32) {
        double t = sh[j * KT + lane];
#pragma unroll
        for (int k = 1; k < KT / 32; ++k) t += sh[j * KT + 32 * k + lane];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) {
            out[j * stride] = t;
            __threadfence();  // each writer orders its partial before the block's ticket (last_block)
        }
    }
}

// ------------------------------------------------------------------ SpMV
// The fine operator runs on a sliced ELLPACK copy of the CSR matrix: slices of SL_W = 32 rows,
// one warp per slice, entry e of every row of the slice stored side by side, so that each load
// of the warp is one contiguous 256-byte (values) or 128-byte (columns) access.  Rows are sorted
// by decreasing length within windows of SL_WIN rows before they are cut into slices, so that
// the rows of a slice have nearly equal lengths (padding of a few per cent on a triangle mesh);
// padding entries hold the row itself as column and 0 as value.  Entries keep the CSR order
// within a row, so y_i sums the same products in the same order as a CSR row loop.
constexpr int SL_W = 32, SL_WIN = 256;

// one CTA per window: rank of every row by (decreasing length, increasing index), the window's
// slot order and the length of each slice (its first, longest row)
__global__ void __launch_bounds__(SL_WIN) k_sell_order(const int *rowptr, int n, int *perm, int *slice_len) {
    __shared__ int len[SL_WIN], sorted[SL_WIN];
    const int w0 = blockIdx.x * SL_WIN, cnt = min(SL_WIN, n - w0), t = threadIdx.x;
    len[t] = t < cnt ? rowptr[w0 + t + 1] - rowptr[w0 + t] : -1;
    __syncthreads();
    if (t < cnt) {
        const int lt = len[t];
        int rank = 0;
        for (int u = 0; u < cnt; ++u) rank += (len[u] > lt || (len[u] == lt && u < t)) ? 1 : 0;
        perm[w0 + rank] = w0 + t;
        sorted[rank] = lt;
    }
    __syncthreads();
    if (t < SL_WIN / SL_W && t * SL_W < cnt) slice_len[w0 / SL_W + t] = sorted[t * SL_W];
}

// 32 * slice length per slice (the scan's input)
__global__ void k_sell_sizes(const int *slice_len, int ns, int *sz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ns) sz[i] = SL_W * slice_len[i];
}

__global__ void k_sell_fill(const int *rowptr, const int *col, const double *val, const int *perm,
                            const int *slice_len, const int *slice_ptr, int n, int *scol, double *sval) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int row = perm[k], e0 = rowptr[row], len = rowptr[row + 1] - e0;
    const int base = slice_ptr[k / SL_W] + (k % SL_W), L = slice_len[k / SL_W];
    for (int e = 0; e < L; ++e) {
        scol[base + SL_W * e] = e < len ? col[e0 + e] : row;
        sval[base + SL_W * e] = e < len ? val[e0 + e] : 0.0;
    }
}

int32_t sell_build(ddg_problem *p) {
    ddg_ctx *c = p->ctx;
    cudaStream_t s = p->stream;
    const int n = p->nf;
    const int ns = cdiv(n, SL_W);
    p->n_slices = ns;
    DDG_TRY(dalloc(c, p->a_matrix, &p->sl_perm, std::max(n, 1)));
    DDG_TRY(dalloc(c, p->a_matrix, &p->sl_len, ns + 1));
    DDG_TRY(dalloc(c, p->a_matrix, &p->sl_ptr, ns + 1));
    if (n == 0) return DDG_OK;
    k_sell_order<<<cdiv(n, SL_WIN), SL_WIN, 0, s>>>(p->rowptr, n, p->sl_perm, p->sl_len);
    k_sell_sizes<<<cdiv(ns, 256), 256, 0, s>>>(p->sl_len, ns, p->sl_ptr);
    DDG_LAUNCH_CHECK();
    DDG_CU(cudaMemsetAsync(p->sl_ptr + ns, 0, sizeof(int), s));
    int total = 0;
    DDG_TRY(scan_exclusive(c, p->sl_ptr, p->sl_ptr, ns + 1, &total, s));
    DDG_TRY(dalloc(c, p->a_matrix, &p->sl_col, std::max(total, 1)));
    DDG_TRY(dalloc(c, p->a_matrix, &p->sl_val, std::max(total, 1)));
    k_sell_fill<<<cdiv(n, 256), 256, 0, s>>>(p->rowptr, p->col, p->val, p->sl_perm, p->sl_len, p->sl_ptr, n,
                                            p->sl_col, p->sl_val);
    DDG_LAUNCH_CHECK();
    DDG_LAUNCHES(3);
    return DDG_OK;
}

// y_row = sum_e val_e x[col_e] for the row of slot k: the first eight entries' columns and values
// are loaded under predicates, then their x gathers, so that all of them are in flight at once
__device__ __forceinline__ double sell_row(const int *__restrict__ scol, const double *__restrict__ sval,
                                           const int *__restrict__ slen, const int *__restrict__ sptr,
                                           const double *__restrict__ x, int k) {
    const int L = slen[k / SL_W];
    const int *cp = scol + sptr[k / SL_W] + (k % SL_W);
    const double *vp = sval + sptr[k / SL_W] + (k % SL_W);
    int c[8];
    double v[8], xv[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        c[e] = e < L ? cp[SL_W * e] : 0;
        v[e] = e < L ? vp[SL_W * e] : 0.0;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) xv[e] = e < L ? x[c[e]] : 0.0;
    double acc = 0.0;
#pragma unroll
    for (int e = 0; e < 8; ++e)
        if (e < L) acc += v[e] * xv[e];
    for (int e = 8; e < L; ++e) acc += vp[SL_W * e] * x[cp[SL_W * e]];
    return acc;
}

__global__ void __launch_bounds__(KT) k_spmv(const int *__restrict__ scol, const double *__restrict__ sval,
                                             const int *__restrict__ slen, const int *__restrict__ sptr,
                                             const int *__restrict__ perm, const double *__restrict__ x,
                                             double *__restrict__ y, int n) {
    const int k = blockIdx.x * KT + threadIdx.x;
    if (k >= n) return;
    y[perm[k]] = sell_row(scol, sval, slen, sptr, x, k);
}

int32_t spmv(ddg_problem *p, const double *x, double *y, cudaStream_t s) {
    k_spmv<<<cdiv(p->nf, KT), KT, 0, s>>>(p->sl_col, p->sl_val, p->sl_len, p->sl_ptr, p->sl_perm, x, y, p->nf);
    DDG_LAUNCH_CHECK();
    return DDG_OK;
}

// ------------------------------------------------------------------ preconditioner pieces
__global__ void __launch_bounds__(KT) k_restrict(const int *sub_ptr, const int *sub_idx, const double *inv_mult,
                                                 const double *r, double *s_out, double *y_out, const int *stop) {
    __shared__ double sh[2 * KT];
    __shared__ double tot[2];
    if (stop && *stop) return;
    int i = blockIdx.x;
    double ss = 0.0, yy = 0.0;
    for (int q = sub_ptr[i] + threadIdx.x; q < sub_ptr[i + 1]; q += KT) {
        int j = sub_idx[q];
        double v = r[j];
        ss += v * v;
        yy += v * inv_mult[j];
    }
    const double v[2] = {ss, yy};
    block_parts<2>(v, 2, sh, tot, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        s_out[i] = sqrt(tot[0]);
        y_out[i] = tot[1];
    }
}

// w = A0inv y, one warp per row
__global__ void k_coarse_gemv(const double *Ainv, const double *y, double *w, int K, const int *stop) {
    if (stop && *stop) return;
    int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (row >= K) return;
    const double *a = Ainv + (long long)row * K;
    double acc = 0.0;
    for (int c = lane; c < K; c += 32) acc += a[c] * y[c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) w[row] = acc;
}

__global__ void __launch_bounds__(KT) k_prolong(const int *mptr, const int *midx, const int *inv_pos,
                                                const double *inv_mult, const double *corr, const double *w, int nf,
                                                int coarse, int pou, double *z, const int *stop) {
    if (stop && *stop) return;
    int j = blockIdx.x * KT + threadIdx.x;
    if (j >= nf) return;
    const double inv_m = inv_mult[j];
    double acc = 0.0;
    int q0 = mptr[j], q1 = mptr[j + 1];
    if (coarse)
        for (int q = q0; q < q1; ++q) acc += inv_m * w[midx[q]];
    for (int q = q0; q < q1; ++q) {
        double c = corr[inv_pos[q]];
        acc += pou ? c * inv_m : c;
    }
    z[j] = acc;
}

__global__ void k_copy(const double *a, double *b, int n, const int *stop) {
    if (stop && *stop) return;
    int i = blockIdx.x * KT + threadIdx.x;
    if (i < n) b[i] = a[i];
}

// records an event; inside a stream capture it becomes an event-record node that
// records each time the graph runs (a plain record would only be a dependency)
static cudaError_t record_event(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t err = cudaStreamIsCapturing(s, &cs);
    if (err != cudaSuccess) return err;
    return cudaEventRecordWithFlags(e, s, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                                : cudaEventRecordDefault);
}

// the preconditioner in three parts: restriction (+ coarse solve), local solves, gluing
static int32_t precond_pre(ddg_problem *p, const double *r, cudaStream_t s, const int *stop, bool prolong, int *nl) {
    const int K = p->K;
    k_restrict<<<K, KT, 0, s>>>(p->sub_ptr, p->sub_idx, p->inv_mult, r, p->s, p->y, stop);
    DDG_LAUNCH_CHECK();
    ++*nl;
    if ((p->flags & DDG_COARSE) && prolong) {
        k_coarse_gemv<<<cdiv(K, 8), 256, 0, s>>>(p->A0inv, p->y, p->wc, K, stop);
        DDG_LAUNCH_CHECK();
        ++*nl;
    }
    return DDG_OK;
}

static int32_t precond_post(ddg_problem *p, double *z, cudaStream_t s, const int *stop, int *nl) {
    const bool coarse = (p->flags & DDG_COARSE) != 0;
    k_prolong<<<cdiv(p->nf, KT), KT, 0, s>>>(p->mem_ptr, p->mem_idx, p->inv_pos, p->inv_mult, p->corr, p->wc,
                                             p->nf, coarse ? 1 : 0, (p->flags & DDG_POU_PROLONG) ? 1 : 0, z, stop);
    DDG_LAUNCH_CHECK();
    ++*nl;
    return DDG_OK;
}

// launches the preconditioner's kernels; ev_local (optional) brackets the local-solve kernel;
// *launches (optional) is increased by the number of kernels launched
static int32_t precond_core(ddg_problem *p, const double *r, double *z, cudaStream_t s, const int *stop,
                            bool prolong, cudaEvent_t *ev_local = nullptr, int *launches = nullptr) {
    int nl = 0;
    if (p->kind == DDG_NONE) {
        if (prolong) {
            k_copy<<<cdiv(p->nf, KT), KT, 0, s>>>(r, z, p->nf, stop);
            DDG_LAUNCH_CHECK();
            nl = 1;
        }
        if (launches) *launches += nl;
        return DDG_OK;
    }
    DDG_TRY(precond_pre(p, r, s, stop, prolong, &nl));
    if (ev_local) DDG_CU(record_event(ev_local[0], s));
    if (p->kind == DDG_DDM_GNN) {
        DDG_TRY(dss_launch_args(p, r, stop, s));
    } else {
        DDG_TRY(lu_apply_launch(p, r, stop, s));
    }
    if (ev_local) DDG_CU(record_event(ev_local[1], s));
    ++nl;
    if (prolong) DDG_TRY(precond_post(p, z, s, stop, &nl));
    if (launches) *launches += nl;
    return DDG_OK;
}

int32_t precond_apply(ddg_problem *p, const double *r, double *z, cudaStream_t s, bool corrections_only,
                      double *corr_out, double *s_out) {
    DDG_TRY(precond_core(p, r, z, s, nullptr, !corrections_only));
    if (corrections_only && p->kind != DDG_NONE) {
        DDG_CU(cudaMemcpyAsync(corr_out, p->corr, sizeof(double) * p->sum_k, cudaMemcpyDeviceToDevice, s));
        DDG_CU(cudaMemcpyAsync(s_out, p->s, sizeof(double) * p->K, cudaMemcpyDeviceToDevice, s));
    }
    return DDG_OK;
}

// Picks the fastest GNN schedule for this decomposition by timing each on the
// right-hand side: 0 = one persistent launch per application; 1 = one launch
// per block, one CTA per graph, weights in the constant bank; 2 = as 1 with
// the graphs cut into chunks of at most 2T nodes (T = 128, 192, 256); 3 = the
// chunks of 2 with composed weights, packed two-lane FP32 and message-sorted nodes;
// 4 = chunks of at most 128 own nodes with the per-node matrix products on the tensor
// cores through tensor memory (tcgen05, dss_tc.cu); 5 = the generic kernel for any latent
// size d in {5, 10, 20} (dss_d.cu), the only schedule for d != 10; 6 = schedule 4's chunks
// with the per-node products as warp-synchronous tensor-core MMAs (dss_mma.cu).
// DDG_GNN_SCHEDULE = 0..6 (and DDG_GNN_CHUNK_T = 128/192/256 for schedule 2,
// 128/256 for schedule 3) forces one.
// The choice is cached in the context per decomposition shape class, so a stream
// of requests of similar sizes tunes once.
int32_t dss_autotune(ddg_problem *p) {
    const char *env = getenv("DDG_GNN_SCHEDULE");
    const char *envT = getenv("DDG_GNN_CHUNK_T");
    // latent sizes other than the compiled d = 10 (or schedule 5 forced): the generic schedule
    if (p->model->d != DSS_D || (env && env[0] == '5' && env[1] == 0)) {
        p->dss_sched = 5;
        return chunk_build(p, DSS_D_CHUNK_T);
    }
    if (env && ((env[0] >= '0' && env[0] <= '4') || env[0] == '6') && env[1] == 0) {
        p->dss_sched = env[0] - '0';
        if (p->dss_sched < 2 && !p->dss_whole_graph) {
            set_error("GNN schedules 0 and 1 need every local graph in one CTA; use 2 or 3");
            return DDG_TOO_LARGE;
        }
        if (p->dss_sched == 2) DDG_TRY(chunk_build(p, envT ? atoi(envT) : 192));
        if (p->dss_sched == 3) DDG_TRY(chunk_build_global(p, envT ? atoi(envT) : 128, false));
        if (p->dss_sched == 4 || p->dss_sched == 6) DDG_TRY(chunk_build_global(p, TC_T, true));
        return DDG_OK;
    }
    const long long cls_K = (long long)std::floor(4.0 * std::log2((double)p->K));
    const long long cls_n = p->sum_loc / ((long long)p->K * 64);
    const long long cls_m = p->max_loc / 128;
    {
        int cached = -1, cachedT = 0;
        {
            std::lock_guard<std::mutex> lock(p->ctx->tune_mu);
            for (const auto &t : p->ctx->tuned)
                if (t.K == cls_K && t.nodes == cls_n && t.max_loc == cls_m && (t.sched >= 2 || p->dss_whole_graph)) {
                    cached = t.sched;
                    cachedT = t.T;
                }
        }
        if (cached >= 0) {
            p->dss_sched = cached;
            if (cached == 2) DDG_TRY(chunk_build(p, cachedT));
            if (cached == 3) DDG_TRY(chunk_build_global(p, cachedT, false));
            if (cached == 4 || cached == 6) DDG_TRY(chunk_build_global(p, TC_T, true));
            return DDG_OK;
        }
    }
    cudaStream_t s = p->stream;
    cudaEvent_t e0, e1;
    DDG_CU(cudaEventCreate(&e0));
    DDG_CU(cudaEventCreate(&e1));
    float best = 1e30f;
    int pick = 0, pickT = 0;
    const int cands[9][2] = {{0, 0}, {1, 0}, {2, 128}, {2, 192}, {2, 256}, {3, 128}, {3, 256}, {4, TC_T}, {6, TC_T}};
    for (const auto &cd : cands) {
        if (cd[0] < 2 && !p->dss_whole_graph) continue;
        p->dss_sched = cd[0];
        if (cd[0] == 2) DDG_TRY(chunk_build(p, cd[1]));
        if (cd[0] == 3) DDG_TRY(chunk_build_global(p, cd[1], false));
        if (cd[0] >= 4 && !p->chunk.tc) DDG_TRY(chunk_build_global(p, cd[1], true));  // 4 and 6 share one plan
        DDG_TRY(precond_core(p, p->b, nullptr, s, nullptr, false));
        DDG_CU(cudaEventRecord(e0, s));
        for (int rep = 0; rep < 2; ++rep) DDG_TRY(precond_core(p, p->b, nullptr, s, nullptr, false));
        DDG_CU(cudaEventRecord(e1, s));
        DDG_CU(cudaEventSynchronize(e1));
        float ms = 0.f;
        DDG_CU(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
            best = ms;
            pick = cd[0];
            pickT = cd[1];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->dss_sched = pick;
    if (pick >= 2) {
        if (p->chunk.T != pickT || p->chunk.global != (pick >= 3) || p->chunk.tc != (pick >= 4))
            DDG_TRY(pick >= 3 ? chunk_build_global(p, pickT, pick >= 4) : chunk_build(p, pickT));
    } else {
        chunk_free(p);
    }
    {
        std::lock_guard<std::mutex> lock(p->ctx->tune_mu);
        p->ctx->tuned.push_back({cls_K, cls_n, cls_m, pick, pickT});
    }
    return check_status(p, "GNN schedule selection");
}

// ------------------------------------------------------------------ FCG kernels
// Each reduction writes one partial per block; the last block to finish (ticket
// counter, reset by that block) sums the partials in block order and derives the
// iteration's scalars, so a solve stays bitwise reproducible without extra launches.
struct Window {
    int W;            // directions to orthogonalise against
    int slot[MAXM];   // their ring slots, oldest first
    int snew;         // slot of the new direction
};

__device__ __forceinline__ bool last_block(int *ticket) {
    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int t = atomicAdd(reinterpret_cast<unsigned int *>(ticket), 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// sum of part[0..n) by one warp in a fixed order (valid in every lane)
__device__ __forceinline__ double warp_sum_parts(const double *__restrict__ part, int n, int lane) {
    double v = 0.0;
#pragma unroll 8
    for (int b = lane; b < n; b += 32) v += part[b];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(KT) k_dot(const double *a, const double *b, int n, double *part) {
    __shared__ double sh[32];
    double v = 0.0;
    for (long long i = (long long)blockIdx.x * KT + threadIdx.x; i < n; i += (long long)RB * KT) v += a[i] * b[i];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// d_j = z . Q[slot_j]; the last block forms beta_j = d_j / (p_j . q_j)
__global__ void __launch_bounds__(KT, 4) k_multidot(const double *z, const double *Q, long long ld, Window win, int n,
                                                    double *part, double *scal, int *flag) {
    __shared__ double sh[MAXM * KT];
    if (flag[F_STOP]) return;
    double acc[MAXM];
#pragma unroll
    for (int j = 0; j < MAXM; ++j) acc[j] = 0.0;
    for (long long i = (long long)blockIdx.x * KT + threadIdx.x; i < n; i += (long long)gridDim.x * KT) {
        double zi = z[i];
#pragma unroll
        for (int j = 0; j < MAXM; ++j)
            if (j < win.W) acc[j] += zi * Q[win.slot[j] * ld + i];
    }
    block_parts<MAXM>(acc, win.W, sh, part + blockIdx.x, RB);
    if (last_block(&flag[F_T_MD])) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int j = warp; j < win.W; j += KT / 32) {
            double d = warp_sum_parts(part + j * RB, gridDim.x, lane);
            if (lane == 0) scal[S_BETA + j] = d / scal[S_PQ + win.slot[j]];
        }
        if (threadIdx.x == 0) flag[F_T_MD] = 0;
    }
}

// P[snew] = z - sum_j beta_j P[slot_j]  (P[snew] may be one of the P[slot_j]: read before write, same index)
__global__ void __launch_bounds__(KT, 4) k_pupdate(const double *z, double *P, long long ld, Window win, int n,
                                                   const double *scal, const int *flag) {
    if (flag[F_STOP]) return;
    __shared__ double beta[MAXM];
    if (threadIdx.x < MAXM) beta[threadIdx.x] = threadIdx.x < win.W ? scal[S_BETA + threadIdx.x] : 0.0;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * KT + threadIdx.x; i < n; i += (long long)gridDim.x * KT) {
        double v = z[i];
#pragma unroll
        for (int j = 0; j < MAXM; ++j)
            if (j < win.W) v -= beta[j] * P[win.slot[j] * ld + i];
        P[win.snew * ld + i] = v;
    }
}

// q = A p with the partial dots p.q and p.r, slots of the sliced ELLPACK matrix strided over
// the grid (up to eight CTAs per SM, a few rows per thread); the last block forms
// alpha = (p.r) / (p.q)
__global__ void __launch_bounds__(KT) k_spmv_fcg(const int *__restrict__ scol, const double *__restrict__ sval,
                                                 const int *__restrict__ slen, const int *__restrict__ sptr,
                                                 const int *__restrict__ perm, const double *__restrict__ p,
                                                 double *__restrict__ q, int n, const double *__restrict__ r,
                                                 double *part, Window win, double *scal, int *flag) {
    __shared__ double sh[2 * KT];
    __shared__ double tot[2];
    if (flag[F_STOP]) return;
    double d[2] = {0.0, 0.0};  // p.q, p.r
    for (int k = blockIdx.x * KT + threadIdx.x; k < n; k += gridDim.x * KT) {
        const double acc = sell_row(scol, sval, slen, sptr, p, k);
        const int i = perm[k];
        q[i] = acc;
        const double pi = p[i];
        d[0] += pi * acc;
        d[1] += pi * r[i];
    }
    block_parts<2>(d, 2, sh, part + blockIdx.x, gridDim.x);
    if (last_block(&flag[F_T_SP])) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (warp < 2) {
            const double t = warp_sum_parts(part + warp * gridDim.x, gridDim.x, lane);
            if (lane == 0) tot[warp] = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double spq = tot[0], spr = tot[1];
            const double al = spr / spq;
            if (!(spq > 0.0) || !isfinite(al)) {
                flag[F_STOP] = 2;
            } else {
                scal[S_PQ + win.snew] = spq;
                scal[S_ALPHA] = al;
            }
            flag[F_T_SP] = 0;
        }
    }
}

// x += alpha p; r -= alpha q; the last block forms |r| / |b| and raises the stop flag
__global__ void __launch_bounds__(KT) k_xr(double *x, double *r, const double *p, const double *q, int n,
                                           double *scal, double *part, int *flag, double tol, double *hist,
                                           int hist_cap) {
    __shared__ double sh[KT];
    if (flag[F_STOP]) return;
    double al = scal[S_ALPHA];
    double v[1] = {0.0};
    for (long long i = (long long)blockIdx.x * KT + threadIdx.x; i < n; i += (long long)gridDim.x * KT) {
        x[i] += al * p[i];
        double ri = r[i] - al * q[i];
        r[i] = ri;
        v[0] += ri * ri;
    }
    block_parts<1>(v, 1, sh, part + blockIdx.x, 0);
    if (last_block(&flag[F_T_XR]) && threadIdx.x < 32) {
        const double rr = warp_sum_parts(part, gridDim.x, threadIdx.x);
        if (threadIdx.x == 0) {
            const double rel = sqrt(rr) / scal[S_BNORM];
            scal[S_REL] = rel;
            if (hist && flag[F_ITERS] < hist_cap) hist[flag[F_ITERS]] = rel;
            flag[F_ITERS] += 1;
            if (!isfinite(rel)) flag[F_STOP] = 2;
            else if (rel < tol) flag[F_STOP] = 1;
            flag[F_T_XR] = 0;
        }
    }
}

// Before the first iteration.  A zero right-hand side has the solution u = 0, so the
// solve ends there with zero iterations (whatever the start vector); a start vector whose
// residual already meets the tolerance ends it the same way.  Without this check both
// cases would reach p.q = 0 in the first step and read as a breakdown.
__global__ void k_initial_check(double *x, int n, double *scal, int *flag, double tol, int r0_is_b) {
    const double bn = scal[S_BNORM];
    if (bn == 0.0)
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
            x[i] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double rel = bn == 0.0 ? 0.0 : (r0_is_b ? 1.0 : scal[S_R0] / bn);
        scal[S_REL] = rel;
        if (bn == 0.0 || rel < tol) flag[F_STOP] = 1;
    }
}

__global__ void k_sumsq_final(const double *part, int nb, double *out) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[b];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) *out = sqrt(v);
}

__global__ void k_residual(const double *b, const double *Ax, double *res, int n) {
    int i = blockIdx.x * KT + threadIdx.x;
    if (i < n) res[i] = b[i] - Ax[i];
}

__global__ void k_full_solution(const double *x, const double *g, const int *free_id, int n, double *u) {
    int a = blockIdx.x * KT + threadIdx.x;
    if (a >= n) return;
    int f = free_id[a];
    u[a] = f >= 0 ? x[f] : g[a];
}

static int32_t norm2(ddg_problem *p, const double *v, double *out_dev, cudaStream_t s) {
    k_dot<<<RB, KT, 0, s>>>(v, v, p->nf, p->kpart);
    DDG_LAUNCH_CHECK();
    k_sumsq_final<<<1, KT, 0, s>>>(p->kpart, RB, out_dev);
    DDG_LAUNCH_CHECK();
    return DDG_OK;
}

// One flexible-CG solve as a resumable state machine: begin() sets the state up,
// launch_batch() queues the next few iterations (direct launches while the
// direction window grows, then replays of a captured period) followed by an
// asynchronous copy of the stop flag, check() tells (blocking or not) whether
// that batch has finished and whether the solve is over, end() computes the
// true residual and the report.  fcg_solve() drives it to completion; the
// request scheduler interleaves many of them.
struct FcgRun {
    ddg_problem *p = nullptr;
    cudaStream_t s = nullptr;
    double rtol = 0.0;
    int max_iter = 0, m = 0, nf = 0, L = 0, nb_spmv = 0;
    int G = 1;  // grid of the reducing FCG kernels (multi-dot, SpMV with its dots, x/r update)
    long long ld = 0, off_sp = 0, off_rr = 0;
    double *record = nullptr;
    double *x = nullptr, *r = nullptr, *z = nullptr, *P = nullptr, *Q = nullptr, *scal = nullptr, *part = nullptr;
    int *flag = nullptr;
    int *hflag = nullptr;  // pinned copy of the flags
    std::vector<cudaEvent_t> ev;
    cudaEvent_t e0 = nullptr, e1 = nullptr, batch_done = nullptr;
    double pre_ms = 0.0, loc_ms = 0.0;
    int loc_launches = 0, loc_applies = 0, launches = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int per_launches = 0, per_loc_launches = 0, per_loc_applies = 0, per_global = 0;
    bool use_graph = true;
    int it = 0, in_flight = 0;

    ~FcgRun() { release(); }

    void release() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
        for (auto &e : ev) cudaEventDestroy(e);
        ev.clear();
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (batch_done) cudaEventDestroy(batch_done);
        e0 = e1 = batch_done = nullptr;
        hflag = nullptr;  // owned by the problem
    }

    void drain(int cnt) {
        for (int q = 0; q < cnt; ++q) {
            float a = 0.f, b = 0.f;
            if (cudaEventElapsedTime(&a, ev[4 * q], ev[4 * q + 1]) != cudaSuccess) a = 0.f;
            if (p->kind != DDG_NONE && cudaEventElapsedTime(&b, ev[4 * q + 2], ev[4 * q + 3]) != cudaSuccess) b = 0.f;
            cudaGetLastError();
            pre_ms += a;
            loc_ms += b;
        }
    }

    int32_t begin(ddg_problem *pp, const double *x0, double rtol_, int max_iter_, int m_, double *record_) {
        p = pp;
        s = p->stream;
        rtol = rtol_;
        max_iter = max_iter_;
        m = m_;
        record = record_;
        nf = p->nf;
        ddg_ctx *c = p->ctx;
        if (m < 1 || m > MAXM) {
            set_error("m_trunc must be in [1, 16]");
            return DDG_INVALID_ARG;
        }
        if (p->kr_m != m) {
            dfree_all(c, p->a_kry);
            p->kr_m = 0;
        }
        if (p->kr_m == 0) {
            DDG_TRY(dalloc(c, p->a_kry, &p->kx, nf));
            DDG_TRY(dalloc(c, p->a_kry, &p->kr, nf));
            DDG_TRY(dalloc(c, p->a_kry, &p->kz, std::max(nf, p->n)));
            DDG_TRY(dalloc(c, p->a_kry, &p->kP, (size_t)m * nf));
            DDG_TRY(dalloc(c, p->a_kry, &p->kQ, (size_t)m * nf));
            DDG_TRY(dalloc(c, p->a_kry, &p->kscal, S_COUNT + 8));
            // partials: multidot (MAXM x RB), SpMV dots (2 per row block), |r|^2 (RB)
            DDG_TRY(dalloc(c, p->a_kry, &p->kpart, (size_t)((MAXM + 1) * RB + 2 * cdiv(nf, KT) + 8)));
            DDG_TRY(dalloc(c, p->a_kry, &p->kflag, F_COUNT));
            p->kr_m = m;
        }
        // residual history of the solve (kept for ddg_fcg_history): the first HIST_MAX iterations
        // at most, so that a large max_iter does not reserve device memory it will not use
        const int hist_need = std::min(max_iter, HIST_MAX);
        if (p->khist_cap < hist_need) {
            dfree_all(c, p->a_hist);
            p->khist = nullptr;
            p->khist_cap = 0;
            DDG_TRY(dalloc(c, p->a_hist, &p->khist, (size_t)hist_need));
            p->khist_cap = hist_need;
        }
        p->khist_n = 0;
        x = p->kx; r = p->kr; z = p->kz; P = p->kP; Q = p->kQ; scal = p->kscal; part = p->kpart;
        flag = p->kflag;
        ld = nf;
        if (!p->hflag_pinned) DDG_CU(cudaMallocHost(&p->hflag_pinned, sizeof(int) * F_COUNT));
        hflag = p->hflag_pinned;
        for (int q = 0; q < F_COUNT; ++q) hflag[q] = 0;
        DDG_CU(cudaMemsetAsync(flag, 0, sizeof(int) * F_COUNT, s));
        DDG_CU(cudaMemsetAsync(scal, 0, sizeof(double) * S_COUNT, s));
        if (x0) {  // r0 = b - A x0
            DDG_CU(cudaMemcpyAsync(x, x0, sizeof(double) * nf, cudaMemcpyHostToDevice, s));
            DDG_TRY(spmv(p, x, z, s));
            k_residual<<<cdiv(nf, KT), KT, 0, s>>>(p->b, z, r, nf);
            DDG_LAUNCH_CHECK();
        } else {
            DDG_CU(cudaMemsetAsync(x, 0, sizeof(double) * nf, s));
            DDG_CU(cudaMemcpyAsync(r, p->b, sizeof(double) * nf, cudaMemcpyDeviceToDevice, s));
        }
        DDG_TRY(norm2(p, p->b, scal + S_BNORM, s));
        if (x0) {
            DDG_TRY(norm2(p, r, scal + S_R0, s));
            k_initial_check<<<RB, KT, 0, s>>>(x, nf, scal, flag, rtol, 0);
        } else {
            k_initial_check<<<1, 32, 0, s>>>(x, 0, scal, flag, rtol, 1);
        }
        DDG_LAUNCH_CHECK();
        DDG_CU(cudaEventCreate(&e0));
        DDG_CU(cudaEventCreate(&e1));
        DDG_CU(cudaEventCreateWithFlags(&batch_done, cudaEventDisableTiming));
        L = m * ((POLL + m - 1) / m);  // iterations per captured period: a multiple of m, at least POLL
        ev.resize(4 * std::max(POLL, L));
        for (auto &e : ev) DDG_CU(cudaEventCreate(&e));
        {
            // between one and two CTAs per SM, so that a thread takes several rows and the block
            // sums (FP64) stay a small share; no more CTAs than row blocks
            int sms = 148;
            DDG_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
            long long g = std::min(std::max((long long)cdiv(nf, KT * 8), (long long)sms), 2LL * sms);
            G = (int)std::max(1LL, std::min(g, (long long)cdiv(nf, KT)));
        }
        // the SpMV: up to eight CTAs per SM (its block sums are two per CTA)
        nb_spmv = (int)std::max(1LL, std::min((long long)RB, (long long)cdiv(nf, KT)));
        off_sp = OFF_MD + MAXM * RB;
        off_rr = off_sp + 2LL * nb_spmv;
        use_graph = getenv("DDG_NO_GRAPH") == nullptr && record == nullptr;
        if (record) DDG_CU(cudaMemcpyAsync(record, r, sizeof(double) * nf, cudaMemcpyDeviceToDevice, s));
        DDG_CU(cudaEventRecord(e0, s));
        it = 0;
        in_flight = 0;
        return DDG_OK;
    }

    // ---- fused-step mode (request loop): the caller runs the local GNN solves of several
    // problems in one launch between group_pre and group_post of one iteration each
    int32_t group_pre() {
        int nl = 0;
        DDG_TRY(precond_pre(p, r, s, flag, true, &nl));
        launches += nl + 1;  // + this problem's share of the fused GNN launches, counted once per step
        ++loc_applies;
        return DDG_OK;
    }

    int32_t group_post() {
        const int iter = it;
        Window win{};
        win.W = std::min(iter, m);
        for (int j = 0; j < win.W; ++j) win.slot[j] = (iter - win.W + j) % m;
        win.snew = iter % m;
        int nl = 0;
        DDG_TRY(precond_post(p, z, s, flag, &nl));
        DDG_TRY(fcg_kernels(win, nl));
        launches += nl;
        ++it;
        ++group_since_mark;
        return DDG_OK;
    }

    int32_t group_mark() {  // queue the flag copy whose completion check() observes
        DDG_CU(cudaMemcpyAsync(hflag, flag, sizeof(int) * F_COUNT, cudaMemcpyDeviceToHost, s));
        DDG_CU(cudaEventRecord(batch_done, s));
        in_flight = 0;
        group_since_mark = 0;
        return DDG_OK;
    }
    int group_since_mark = 0;

    // the four FCG kernels of one iteration after z = M^-1 r
    int32_t fcg_kernels(const Window &win, int &nl) {
        double *pn = P + win.snew * ld, *qn = Q + win.snew * ld;
        if (win.W > 0) {
            k_multidot<<<G, KT, 0, s>>>(z, Q, ld, win, nf, part + OFF_MD, scal, flag);
            ++nl;
            DDG_LAUNCHES(1);
        }
        k_pupdate<<<PUG, KT, 0, s>>>(z, P, ld, win, nf, scal, flag);
        k_spmv_fcg<<<nb_spmv, KT, 0, s>>>(p->sl_col, p->sl_val, p->sl_len, p->sl_ptr, p->sl_perm, pn, qn, nf, r,
                                          part + off_sp, win, scal, flag);
        k_xr<<<G, KT, 0, s>>>(x, r, pn, qn, nf, scal, part + off_rr, flag, rtol, p->khist, p->khist_cap);
        nl += 3;
        DDG_LAUNCHES(3);
        return DDG_OK;
    }

    // launches one FCG iteration; q indexes the iteration's event slot
    int32_t launch_iter(int iter, int q) {
        Window win{};
        win.W = std::min(iter, m);
        for (int j = 0; j < win.W; ++j) win.slot[j] = (iter - win.W + j) % m;
        win.snew = iter % m;
        cudaEvent_t *evq = ev.data() + 4 * q;
        DDG_CU(record_event(evq[0], s));
        DDG_TRY(precond_core(p, r, z, s, flag, true, p->kind != DDG_NONE ? evq + 2 : nullptr, &launches));
        DDG_CU(record_event(evq[1], s));
        if (p->kind != DDG_NONE) {
            ++loc_applies;
            loc_launches += (p->kind == DDG_DDM_GNN && p->dss_sched >= 1) ? p->model->kbar : 1;
        }
        int nl = 0;
        DDG_TRY(fcg_kernels(win, nl));
        launches += nl;
        if (record)
            DDG_CU(cudaMemcpyAsync(record + (size_t)(iter + 1) * nf, r, sizeof(double) * nf, cudaMemcpyDeviceToDevice, s));
        return DDG_OK;
    }

    // The first m iterations grow the direction window; from iteration m on the
    // ring slots repeat with period m, so one period is captured as a CUDA graph
    // and replayed.  Queues one batch and the copy of the stop flag behind it.
    // Captures one period of L iterations (ring windows of iterations m .. m + L - 1, the same for
    // every period that starts at a multiple of m) and instantiates it.  The launches recorded
    // during the capture are not executions: they are taken back out of the counters, and every
    // replay adds them.
    int32_t capture_period() {
        const int l0 = launches, ll0 = loc_launches, la0 = loc_applies;
        const unsigned long long g0 = launch_count();
        DDG_CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int32_t st = DDG_OK;
        for (int q = 0; q < L && st == DDG_OK; ++q) st = launch_iter(m + q, q);
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (st != DDG_OK) return st;
        DDG_CU(ce);
        DDG_CU(cudaGraphInstantiate(&gexec, graph, 0));
        per_launches = launches - l0;
        per_loc_launches = loc_launches - ll0;
        per_loc_applies = loc_applies - la0;
        per_global = (int)(launch_count() - g0);
        launches = l0;
        loc_launches = ll0;
        loc_applies = la0;
        note_launches(-per_global);
        return DDG_OK;
    }

    int32_t launch_batch() {
        if (gexec && it >= m && it % m == 0 && max_iter - it >= L) {
            launches += per_launches;
            loc_launches += per_loc_launches;
            loc_applies += per_loc_applies;
            note_launches(per_global);
            DDG_CU(cudaGraphLaunch(gexec, s));
            it += L;
            in_flight = L;
        } else {
            int n = 0;
            do {
                DDG_TRY(launch_iter(it, n));
                ++it;
                ++n;
            } while (n < POLL && it < max_iter && !(use_graph && it == m));
            in_flight = n;
        }
        DDG_CU(cudaMemcpyAsync(hflag, flag, sizeof(int) * F_COUNT, cudaMemcpyDeviceToHost, s));
        DDG_CU(cudaEventRecord(batch_done, s));
        // with this batch queued, the host captures the replayed period while the GPU works on
        // it, instead of leaving the GPU idle for the capture when iteration m is reached
        if (use_graph && !gexec && max_iter - m >= L) DDG_TRY(capture_period());
        return DDG_OK;
    }

    // *ready: the queued batch has finished; *done: the solve is over
    int32_t check(bool blocking, bool *ready, bool *done) {
        if (blocking) {
            DDG_CU(cudaEventSynchronize(batch_done));
        } else {
            cudaError_t q = cudaEventQuery(batch_done);
            if (q == cudaErrorNotReady) {
                *ready = false;
                *done = false;
                return DDG_OK;
            }
            DDG_CU(q);
        }
        *ready = true;
        drain(in_flight);
        in_flight = 0;
        *done = hflag[F_STOP] != 0 || it >= max_iter;
        return DDG_OK;
    }

    int32_t end(double *x_host, ddg_solve_report *rep) {
        DDG_CU(cudaEventRecord(e1, s));
        DDG_CU(cudaMemcpyAsync(hflag, flag, sizeof(int) * F_COUNT, cudaMemcpyDeviceToHost, s));
        double hs[S_COUNT];
        DDG_CU(cudaMemcpyAsync(hs, scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s));
        // true residual |b - A x| / |b|
        DDG_TRY(spmv(p, x, z, s));
        k_residual<<<cdiv(nf, KT), KT, 0, s>>>(p->b, z, z, nf);
        DDG_LAUNCH_CHECK();
        double *tr = scal + S_COUNT;
        DDG_TRY(norm2(p, z, tr, s));
        double htr = 0.0;
        DDG_CU(cudaMemcpyAsync(&htr, tr, sizeof(double), cudaMemcpyDeviceToHost, s));
        if (x_host) {
            k_full_solution<<<cdiv(p->n, KT), KT, 0, s>>>(x, p->g, p->free_id, p->n, z);
            DDG_LAUNCH_CHECK();
            DDG_CU(cudaMemcpyAsync(x_host, z, sizeof(double) * p->n, cudaMemcpyDeviceToHost, s));
        }
        DDG_CU(cudaStreamSynchronize(s));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ddg_solve_report rp{};
        rp.iterations = hflag[F_ITERS];
        p->khist_n = std::min(hflag[F_ITERS], p->khist_cap);
        rp.rel_residual = hs[S_REL];
        rp.true_rel_residual = hs[S_BNORM] > 0.0 ? htr / hs[S_BNORM] : 0.0;  // b = 0: u = 0 is exact
        rp.solve_ms = ms;
        rp.precond_ms = pre_ms;
        rp.local_ms = loc_ms;
        rp.local_launches = loc_launches;
        rp.launches = launches;
        rp.local_applies = loc_applies;
        rp.gnn_schedule = p->kind == DDG_DDM_GNN ? p->dss_sched : -1;
        rp.gnn_chunk_t = (p->kind == DDG_DDM_GNN && p->dss_sched >= 2) ? p->chunk.T : 0;
        rp.status = hflag[F_STOP] == 1 ? DDG_OK : (hflag[F_STOP] == 2 ? DDG_BREAKDOWN : DDG_NOT_CONVERGED);
        // a kernel that gave up a bounded wait (or met another device-side error) overrides the outcome
        const int32_t dev = check_status(p, "FCG solve");
        if (dev != DDG_OK) rp.status = dev;
        if (rep) *rep = rp;
        release();
        if (dev != DDG_OK) return dev;
        if (rp.status == DDG_BREAKDOWN) set_error("FCG breakdown: p.q <= 0 or a non-finite scalar");
        if (rp.status == DDG_NOT_CONVERGED) set_error("FCG reached max_iter");
        return rp.status;
    }
};

int32_t fcg_group_pre(FcgRun *r) { return r->group_pre(); }
int32_t fcg_group_post(FcgRun *r) { return r->group_post(); }
int32_t fcg_group_mark(FcgRun *r) { return r->group_mark(); }
int fcg_group_since_mark(const FcgRun *r) { return r->group_since_mark; }
int fcg_iterations_launched(const FcgRun *r) { return r->it; }
int fcg_max_iter(const FcgRun *r) { return r->max_iter; }
const double *fcg_residual(const FcgRun *r) { return r->r; }
const int *fcg_flag(const FcgRun *r) { return r->flag; }

FcgRun *fcg_new() { return new FcgRun(); }
void fcg_delete(FcgRun *r) { delete r; }
int32_t fcg_begin(FcgRun *r, ddg_problem *p, const double *x0, double rtol, int max_iter, int m) {
    return r->begin(p, x0, rtol, max_iter, m, nullptr);
}
int32_t fcg_launch_batch(FcgRun *r) { return r->launch_batch(); }
int32_t fcg_check(FcgRun *r, bool blocking, bool *ready, bool *done) { return r->check(blocking, ready, done); }
int32_t fcg_end(FcgRun *r, double *x_host, ddg_solve_report *rep) { return r->end(x_host, rep); }

int32_t fcg_solve(ddg_problem *p, const double *x0, double rtol, int max_iter, int m, double *x_host,
                  ddg_solve_report *rep, double *record) {
    FcgRun run;
    DDG_TRY(run.begin(p, x0, rtol, max_iter, m, record));
    bool ready = false, done = false;
    while (!done) {
        DDG_TRY(run.launch_batch());
        DDG_TRY(run.check(true, &ready, &done));
    }
    return run.end(x_host, rep);
}

// Runs PCG (FCG with m = 1) with the current preconditioner for at most iters - 1
// iterations and stores r_0, r_1, ... in record[iters][n_free]; returns how many
// residuals were stored (the solve may converge earlier).
int32_t fcg_solve_record(ddg_problem *p, int iters, double *record, int *stored) {
    ddg_solve_report rep{};
    int32_t st = fcg_solve(p, nullptr, 1e-14, iters - 1, 1, nullptr, &rep, record);
    if (st != DDG_OK && st != DDG_NOT_CONVERGED && st != DDG_BREAKDOWN) return st;
    *stored = std::min(iters, rep.iterations + 1);
    clear_error();
    return DDG_OK;
}

}  // namespace ddg
