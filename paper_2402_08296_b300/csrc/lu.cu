// DDM-LU local solves (Eq. 7; Section IV-C's exact-solve comparator): every
// R_i A R_i^T is factorised once by FP64 band Cholesky and applied by a
// forward and a backward band triangular solve per preconditioner call.
//
// Ordering: the unknowns of a subdomain are renumbered along the longer side
// of their bounding box (ties by local index), which makes the local matrix
// banded with a half-bandwidth of a few times the subdomain's width in nodes.
// Storage per subdomain: row r holds L[r][r-bw .. r] (bw + 1 FP64 values).
#include "ddg_internal.cuh"

#include <algorithm>
#include <cfloat>
#include <climits>

namespace ddg {

constexpr int LU_T = 256;

__device__ __forceinline__ int lower_bound_lu(const int *a, int n, int v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int m = (lo + hi) >> 1;
        if (a[m] < v) lo = m + 1; else hi = m;
    }
    return lo;
}

// band order of the unknowns of subdomain blockIdx.x
__global__ void __launch_bounds__(LU_T) k_lu_order(const int *sub_ptr, const int *sub_idx, const double *xy_free,
                                                   int *lu_perm, int *lu_pos) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double red[4][32];
    const int i = blockIdx.x;
    const int s0 = sub_ptr[i], k = sub_ptr[i + 1] - s0;
    int N = 1;
    while (N < k) N <<= 1;
    double *key = reinterpret_cast<double *>(sm);
    int *idx = reinterpret_cast<int *>(key + N);
    double mnx = DBL_MAX, mxx = -DBL_MAX, mny = DBL_MAX, mxy = -DBL_MAX;
    for (int t = threadIdx.x; t < k; t += LU_T) {
        int f = sub_idx[s0 + t];
        double x = xy_free[2 * f], y = xy_free[2 * f + 1];
        mnx = fmin(mnx, x); mxx = fmax(mxx, x); mny = fmin(mny, y); mxy = fmax(mxy, y);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mnx = fmin(mnx, __shfl_down_sync(0xffffffffu, mnx, o));
        mxx = fmax(mxx, __shfl_down_sync(0xffffffffu, mxx, o));
        mny = fmin(mny, __shfl_down_sync(0xffffffffu, mny, o));
        mxy = fmax(mxy, __shfl_down_sync(0xffffffffu, mxy, o));
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red[0][warp] = mnx; red[1][warp] = mxx; red[2][warp] = mny; red[3][warp] = mxy; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < LU_T / 32; ++w) {
            red[0][0] = fmin(red[0][0], red[0][w]); red[1][0] = fmax(red[1][0], red[1][w]);
            red[2][0] = fmin(red[2][0], red[2][w]); red[3][0] = fmax(red[3][0], red[3][w]);
        }
    }
    __syncthreads();
    const int axis = (red[1][0] - red[0][0]) >= (red[3][0] - red[2][0]) ? 0 : 1;
    for (int t = threadIdx.x; t < N; t += LU_T) {
        if (t < k) {
            key[t] = xy_free[2 * sub_idx[s0 + t] + axis];
            idx[t] = t;
        } else {
            key[t] = DBL_MAX;
            idx[t] = INT_MAX;
        }
    }
    __syncthreads();
    for (int kk = 2; kk <= N; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int q = threadIdx.x; q < N; q += LU_T) {
                int r = q ^ j;
                if (r > q) {
                    bool up = (q & kk) == 0;
                    bool gt = key[q] > key[r] || (key[q] == key[r] && idx[q] > idx[r]);
                    if (gt == up) {
                        double tk = key[q]; key[q] = key[r]; key[r] = tk;
                        int ti = idx[q]; idx[q] = idx[r]; idx[r] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int b = threadIdx.x; b < k; b += LU_T) {
        lu_perm[s0 + b] = idx[b];
        lu_pos[s0 + idx[b]] = b;
    }
}

__global__ void __launch_bounds__(LU_T) k_lu_bw(const int *sub_ptr, const int *sub_idx, const int *rowptr,
                                                const int *col, const int *mptr, const int *midx,
                                                const int *lu_pos, int *bw_out) {
    __shared__ int smax;
    const int i = blockIdx.x;
    const int s0 = sub_ptr[i], k = sub_ptr[i + 1] - s0;
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();
    int m = 0;
    for (int t = threadIdx.x; t < k; t += LU_T) {
        int f = sub_idx[s0 + t];
        int pr = lu_pos[s0 + t];
        for (int e = rowptr[f]; e < rowptr[f + 1]; ++e) {
            int l = col[e];
            bool inside = false;
            for (int q = mptr[l]; q < mptr[l + 1]; ++q) inside |= midx[q] == i;
            if (!inside) continue;
            int tl = lower_bound_lu(sub_idx + s0, k, l);
            m = max(m, abs(pr - lu_pos[s0 + tl]));
        }
    }
    atomicMax(&smax, m);
    __syncthreads();
    if (threadIdx.x == 0) bw_out[i] = smax;
}

__global__ void __launch_bounds__(LU_T) k_lu_fill(const int *sub_ptr, const int *sub_idx, const int *rowptr,
                                                  const int *col, const double *val, const int *mptr,
                                                  const int *midx, const int *lu_pos, const int *bw,
                                                  const long long *off, double *band) {
    const int i = blockIdx.x;
    const int s0 = sub_ptr[i], k = sub_ptr[i + 1] - s0;
    const int w = bw[i] + 1;
    double *B = band + off[i];
    for (long long q = threadIdx.x; q < (long long)k * w; q += LU_T) B[q] = 0.0;
    __syncthreads();
    for (int t = threadIdx.x; t < k; t += LU_T) {
        int f = sub_idx[s0 + t];
        int r = lu_pos[s0 + t];
        for (int e = rowptr[f]; e < rowptr[f + 1]; ++e) {
            int l = col[e];
            bool inside = false;
            for (int q = mptr[l]; q < mptr[l + 1]; ++q) inside |= midx[q] == i;
            if (!inside) continue;
            int c = lu_pos[s0 + lower_bound_lu(sub_idx + s0, k, l)];
            if (c <= r) B[(long long)r * w + (c - r + w - 1)] = val[e];
        }
    }
}

// right-looking band Cholesky, one CTA per subdomain; the diagonal slot of
// every row receives 1 / L[r][r] so that the solves multiply instead of divide
__global__ void __launch_bounds__(LU_T) k_lu_factor(const int *sub_ptr, const int *bw_arr, const long long *off,
                                                    double *band, int *st) {
    __shared__ double dinv;
    __shared__ int bad;
    const int i = blockIdx.x;
    const int k = sub_ptr[i + 1] - sub_ptr[i];
    const int bw = bw_arr[i], w = bw + 1;
    double *B = band + off[i];
    if (threadIdx.x == 0) bad = 0;
    for (int c = 0; c < k; ++c) {
        if (threadIdx.x == 0) {
            double d = B[(long long)c * w + bw];
            if (!(d > 0.0)) {
                bad = 1;
                d = 1.0;
            }
            dinv = 1.0 / sqrt(d);
            B[(long long)c * w + bw] = dinv;
        }
        __syncthreads();
        const int rmax = min(c + bw, k - 1);
        for (int r = c + 1 + threadIdx.x; r <= rmax; r += LU_T) B[(long long)r * w + (c - r + bw)] *= dinv;
        __syncthreads();
        const int span = rmax - c;
        for (int q = threadIdx.x; q < span * span; q += LU_T) {
            int dr = q / span + 1, dq = q % span + 1;
            if (dq <= dr) {
                int r = c + dr, cq = c + dq;
                B[(long long)r * w + (cq - r + bw)] -= B[(long long)r * w + (c - r + bw)] * B[(long long)cq * w + (c - cq + bw)];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && bad) raise_status(st, ST_BAD_INPUT);
}

// forward and backward band solves, one CTA per subdomain, rows in tiles of 32:
// the CTA stages each 32 x 32 diagonal tile of the factor in shared memory with
// coalesced loads, a warp solves it from there, and the whole CTA applies the
// band entries outside it; corr is written in sub_idx order
constexpr int LU_TILE = 32;

// Ds[rr][cc] = L[r0 + rr][r0 + cc] inside the band (diagonal slot: 1 / L_rr), 0 elsewhere
__device__ __forceinline__ void lu_stage_tile(double (*Ds)[LU_TILE + 1], const double *B, int w, int bw, int r0,
                                              int nrow) {
    for (int q = threadIdx.x; q < LU_TILE * LU_TILE; q += LU_T) {
        const int rr = q / LU_TILE, cc = q % LU_TILE;
        double v = 0.0;
        if (rr < nrow && cc <= rr && rr - cc <= bw) v = B[(long long)(r0 + rr) * w + (cc - rr + bw)];
        Ds[rr][cc] = v;
    }
}

__global__ void __launch_bounds__(LU_T) k_lu_apply(const int *sub_ptr, const int *sub_idx, const int *lu_pos,
                                                   const int *bw_arr, const long long *off, const double *band,
                                                   const double *r, const double *s, double *corr, const int *stop) {
    extern __shared__ double yv[];
    __shared__ double Ds[LU_TILE][LU_TILE + 1];
    if (stop && *stop) return;
    const int i = blockIdx.x;
    const int s0 = sub_ptr[i], k = sub_ptr[i + 1] - s0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bw = bw_arr[i], w = bw + 1;
    const double *B = band + off[i];
    if (s[i] == 0.0) {
        for (int t = tid; t < k; t += LU_T) corr[s0 + t] = 0.0;
        return;
    }
    for (int t = tid; t < k; t += LU_T) yv[lu_pos[s0 + t]] = r[sub_idx[s0 + t]];
    __syncthreads();
    // L y = b
    for (int r0 = 0; r0 < k; r0 += LU_TILE) {
        const int nrow = min(LU_TILE, k - r0);
        for (int rr = warp; rr < nrow; rr += LU_T / 32) {
            const int row = r0 + rr;
            const double *Lr = B + (long long)row * w;
            double acc = 0.0;
            for (int c = max(0, row - bw) + lane; c < r0; c += 32) acc += Lr[c - row + bw] * yv[c];
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) yv[row] -= acc;
        }
        lu_stage_tile(Ds, B, w, bw, r0, nrow);
        __syncthreads();
        if (warp == 0) {
            const int row = r0 + lane;
            double y = lane < nrow ? yv[row] : 0.0;
            for (int j = 0; j < nrow; ++j) {
                if (lane == j) y *= Ds[j][j];
                const double xj = __shfl_sync(0xffffffffu, y, j);
                if (lane > j && lane < nrow && lane - j <= bw) y -= Ds[lane][j] * xj;
            }
            if (lane < nrow) yv[row] = y;
        }
        __syncthreads();
    }
    // L^T x = y, tiles from the bottom
    for (int r0 = ((k - 1) / LU_TILE) * LU_TILE; r0 >= 0; r0 -= LU_TILE) {
        const int nrow = min(LU_TILE, k - r0);
        lu_stage_tile(Ds, B, w, bw, r0, nrow);
        __syncthreads();
        if (warp == 0) {
            const int row = r0 + lane;
            double y = lane < nrow ? yv[row] : 0.0;
            const double dinv = lane < nrow ? Ds[lane][lane] : 0.0;
            for (int j = nrow - 1; j >= 0; --j) {
                if (lane == j) y *= dinv;
                const double xj = __shfl_sync(0xffffffffu, y, j);
                if (lane < j && j - lane <= bw) y -= Ds[j][lane] * xj;
            }
            if (lane < nrow) yv[row] = y;
        }
        __syncthreads();
        for (int c = max(0, r0 - bw) + tid; c < r0; c += LU_T) {
            double acc = 0.0;
            for (int qq = 0; qq < nrow; ++qq) {
                const int q = r0 + qq;
                if (q - c <= bw) acc += B[(long long)q * w + (c - q + bw)] * yv[q];
            }
            yv[c] -= acc;
        }
        __syncthreads();
    }
    for (int t = tid; t < k; t += LU_T) corr[s0 + t] = yv[lu_pos[s0 + t]];
}

int32_t lu_build(ddg_problem *p) {
    ddg_ctx *c = p->ctx;
    cudaStream_t s = p->stream;
    const int K = p->K;
    std::vector<int> hp(K + 1);
    DDG_CU(cudaMemcpyAsync(hp.data(), p->sub_ptr, sizeof(int) * (K + 1), cudaMemcpyDeviceToHost, s));
    DDG_CU(cudaStreamSynchronize(s));
    int kmax = 0;
    for (int i = 0; i < K; ++i) kmax = std::max(kmax, hp[i + 1] - hp[i]);
    int N = 1;
    while (N < kmax) N <<= 1;
    size_t order_smem = (size_t)N * (sizeof(double) + sizeof(int));
    if (order_smem > 200 * 1024 || (size_t)kmax * sizeof(double) > 200 * 1024) {
        set_error("subdomain too large for the band factor kernels");
        return DDG_TOO_LARGE;
    }
    DDG_CU(cudaFuncSetAttribute(k_lu_order, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    DDG_CU(cudaFuncSetAttribute(k_lu_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    DDG_TRY(dalloc(c, p->a_pre, &p->lu_perm, p->sum_k));
    DDG_TRY(dalloc(c, p->a_pre, &p->lu_pos, p->sum_k));
    DDG_TRY(dalloc(c, p->a_pre, &p->lu_bw, K));
    DDG_TRY(dalloc(c, p->a_pre, &p->lu_off, K + 1));
    k_lu_order<<<K, LU_T, order_smem, s>>>(p->sub_ptr, p->sub_idx, p->xy_free, p->lu_perm, p->lu_pos);
    DDG_LAUNCH_CHECK();
    k_lu_bw<<<K, LU_T, 0, s>>>(p->sub_ptr, p->sub_idx, p->rowptr, p->col, p->mem_ptr, p->mem_idx, p->lu_pos,
                               p->lu_bw);
    DDG_LAUNCH_CHECK();
    std::vector<int> hb(K);
    DDG_CU(cudaMemcpyAsync(hb.data(), p->lu_bw, sizeof(int) * K, cudaMemcpyDeviceToHost, s));
    DDG_CU(cudaStreamSynchronize(s));
    std::vector<long long> off(K + 1, 0);
    for (int i = 0; i < K; ++i) off[i + 1] = off[i] + (long long)(hp[i + 1] - hp[i]) * (hb[i] + 1);
    DDG_CU(cudaMemcpyAsync(p->lu_off, off.data(), sizeof(long long) * (K + 1), cudaMemcpyHostToDevice, s));
    DDG_TRY(dalloc(c, p->a_pre, &p->lu_band, off[K]));
    k_lu_fill<<<K, LU_T, 0, s>>>(p->sub_ptr, p->sub_idx, p->rowptr, p->col, p->val, p->mem_ptr, p->mem_idx,
                                 p->lu_pos, p->lu_bw, p->lu_off, p->lu_band);
    DDG_LAUNCH_CHECK();
    k_lu_factor<<<K, LU_T, 0, s>>>(p->sub_ptr, p->lu_bw, p->lu_off, p->lu_band, p->d_status);
    DDG_LAUNCH_CHECK();
    DDG_CU(cudaStreamSynchronize(s));
    p->lu_kmax = kmax;
    int32_t r = check_status(p, "band Cholesky");
    if (r == DDG_INVALID_ARG) set_error("a local matrix is not positive definite");
    return r;
}

int32_t lu_apply_launch(ddg_problem *p, const double *r, const int *stop, cudaStream_t s) {
    k_lu_apply<<<p->K, LU_T, sizeof(double) * p->lu_kmax, s>>>(p->sub_ptr, p->sub_idx, p->lu_pos, p->lu_bw,
                                                             p->lu_off, p->lu_band, r, p->s, p->corr, stop);
    DDG_LAUNCH_CHECK();
    return DDG_OK;
}

}  // namespace ddg
