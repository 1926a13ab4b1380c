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

// The solves run in tiles of 32 rows.  Set-up keeps, besides the factor, its transpose in
// the same band storage (row c holds L[c .. c + bw][c], diagonal first) so that the backward
// solve reads rows contiguously too, and the inverse of every 32 x 32 diagonal tile of L
// (lower triangular), so that a tile's triangular solve is one small matrix-vector product
// instead of 32 dependent steps.
constexpr int LU_TILE = 32;
static_assert(LU_T == LU_TILE * 8, "a solve CTA is 32 rows of 8 threads");

__global__ void __launch_bounds__(LU_T) k_lu_transpose(const int *sub_ptr, const int *bw_arr, const long long *off,
                                                       const double *band, double *bandT) {
    const int i = blockIdx.x;
    const int k = sub_ptr[i + 1] - sub_ptr[i];
    const int bw = bw_arr[i], w = bw + 1;
    const double *B = band + off[i];
    double *U = bandT + off[i];
    for (long long qq = threadIdx.x; qq < (long long)k * w; qq += LU_T) {
        const int c = (int)(qq / w), j = (int)(qq % w);  // U[c][c + j] = L[c + j][c]
        const int q = c + j;
        U[qq] = q < k ? B[(long long)q * w + (c - q + bw)] : 0.0;
    }
}

// inverse of every diagonal tile, one warp per subdomain: lane j computes column j by forward
// substitution, x_r = (delta_rj - sum_{m<r} L[r][m] x_m) / L[r][r]; rows and columns past the
// subdomain's end are zero
__global__ void __launch_bounds__(32) k_lu_tinv(const int *sub_ptr, const int *bw_arr, const long long *off,
                                               const long long *toff, const double *band, double *tinv) {
    __shared__ double X[LU_TILE][LU_TILE + 1];
    const int i = blockIdx.x, lane = threadIdx.x;
    const int k = sub_ptr[i + 1] - sub_ptr[i];
    const int bw = bw_arr[i], w = bw + 1;
    const double *B = band + off[i];
    double *T = tinv + toff[i];
    const int nt = (k + LU_TILE - 1) / LU_TILE;
    for (int t = 0; t < nt; ++t) {
        const int r0 = t * LU_TILE, nrow = min(LU_TILE, k - r0);
        for (int r = 0; r < LU_TILE; ++r) {
            double acc = 0.0;
            if (r < nrow && lane < nrow && lane <= r) {
                acc = r == lane ? 1.0 : 0.0;
                const double *Lr = B + (long long)(r0 + r) * w;
                for (int m = max(lane, r - bw); m < r; ++m) acc -= Lr[m - r + bw] * X[m][lane];
                acc *= Lr[bw];  // the diagonal slot holds 1 / L[r][r]
            }
            X[r][lane] = acc;
        }
        for (int r = 0; r < LU_TILE; ++r) T[(long long)t * LU_TILE * LU_TILE + r * LU_TILE + lane] = X[r][lane];
        __syncwarp();
    }
}

// forward and backward band solves, one CTA per subdomain, 8 threads per row of a tile: the
// band entries left of (forward) or below (backward) the tile are summed in parallel, then
// the tile's inverse (or its transpose) is applied; corr is written in sub_idx order
__global__ void __launch_bounds__(LU_T) k_lu_apply(const int *sub_ptr, const int *sub_idx, const int *lu_pos,
                                                   const int *bw_arr, const long long *off, const long long *toff,
                                                   const double *band, const double *bandT, const double *tinv,
                                                   const double *r, const double *s, double *corr, const int *stop) {
    extern __shared__ double yv[];
    __shared__ double rhs[LU_TILE];
    if (stop && *stop) return;
    const int i = blockIdx.x;
    const int s0 = sub_ptr[i], k = sub_ptr[i + 1] - s0;
    const int tid = threadIdx.x, rr = tid >> 3, part = tid & 7;
    const int bw = bw_arr[i], w = bw + 1;
    const double *B = band + off[i], *U = bandT + off[i], *T = tinv + toff[i];
    if (s[i] == 0.0) {
        for (int t = tid; t < k; t += LU_T) corr[s0 + t] = 0.0;
        return;
    }
    for (int t = tid; t < k; t += LU_T) yv[lu_pos[s0 + t]] = r[sub_idx[s0 + t]];
    __syncthreads();
    const int nt = (k + LU_TILE - 1) / LU_TILE;
    // L y = b
    for (int t = 0; t < nt; ++t) {
        const int r0 = t * LU_TILE, nrow = min(LU_TILE, k - r0), row = r0 + rr;
        const double *Tt = T + (long long)t * LU_TILE * LU_TILE;
        double tv[4];  // L_tt^-1 [rr][part + 8 j]: independent of the sums, loaded first
#pragma unroll
        for (int j = 0; j < 4; ++j) tv[j] = rr < nrow ? Tt[rr * LU_TILE + part + 8 * j] : 0.0;
        double acc = 0.0;
        if (rr < nrow) {
            const double *Lr = B + (long long)row * w;
#pragma unroll 4
            for (int c = max(0, row - bw) + part; c < r0; c += 8) acc += Lr[c - row + bw] * yv[c];
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (part == 0 && rr < nrow) rhs[rr] = yv[row] - acc;
        __syncthreads();
        double y = 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (part + 8 * j < nrow) y += tv[j] * rhs[part + 8 * j];
        y += __shfl_xor_sync(0xffffffffu, y, 4);
        y += __shfl_xor_sync(0xffffffffu, y, 2);
        y += __shfl_xor_sync(0xffffffffu, y, 1);
        if (part == 0 && rr < nrow) yv[row] = y;
        __syncthreads();
    }
    // L^T x = y, tiles from the bottom
    for (int t = nt - 1; t >= 0; --t) {
        const int r0 = t * LU_TILE, nrow = min(LU_TILE, k - r0), row = r0 + rr, r1 = r0 + nrow - 1;
        const double *Tt = T + (long long)t * LU_TILE * LU_TILE;
        double tv[4];  // (L_tt^-1)^T [rr][part + 8 j]
#pragma unroll
        for (int j = 0; j < 4; ++j) tv[j] = rr < nrow ? Tt[(part + 8 * j) * LU_TILE + rr] : 0.0;
        double acc = 0.0;
        if (rr < nrow) {
            const double *Ur = U + (long long)row * w;  // Ur[j] = L[row + j][row]
            const int qmax = min(k - 1, row + bw);
#pragma unroll 4
            for (int q = r1 + 1 + part; q <= qmax; q += 8) acc += Ur[q - row] * yv[q];
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (part == 0 && rr < nrow) rhs[rr] = yv[row] - acc;
        __syncthreads();
        double x = 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (part + 8 * j < nrow) x += tv[j] * rhs[part + 8 * j];
        x += __shfl_xor_sync(0xffffffffu, x, 4);
        x += __shfl_xor_sync(0xffffffffu, x, 2);
        x += __shfl_xor_sync(0xffffffffu, x, 1);
        if (part == 0 && rr < nrow) yv[row] = x;
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
    // the transposed band and the diagonal tiles' inverses of the solves
    std::vector<long long> toff(K + 1, 0);
    for (int i = 0; i < K; ++i) toff[i + 1] = toff[i] + (long long)((hp[i + 1] - hp[i] + LU_TILE - 1) / LU_TILE) * LU_TILE * LU_TILE;
    DDG_TRY(dalloc(c, p->a_pre, &p->lu_toff, K + 1));
    DDG_CU(cudaMemcpyAsync(p->lu_toff, toff.data(), sizeof(long long) * (K + 1), cudaMemcpyHostToDevice, s));
    DDG_TRY(dalloc(c, p->a_pre, &p->lu_bandT, off[K]));
    DDG_TRY(dalloc(c, p->a_pre, &p->lu_tinv, toff[K]));
    k_lu_transpose<<<K, LU_T, 0, s>>>(p->sub_ptr, p->lu_bw, p->lu_off, p->lu_band, p->lu_bandT);
    DDG_LAUNCH_CHECK();
    k_lu_tinv<<<K, 32, 0, s>>>(p->sub_ptr, p->lu_bw, p->lu_off, p->lu_toff, p->lu_band, p->lu_tinv);
    DDG_LAUNCH_CHECK();
    DDG_CU(cudaStreamSynchronize(s));
    p->lu_kmax = kmax;
    int32_t r = check_status(p, "band Cholesky");
    if (r == DDG_INVALID_ARG) set_error("a local matrix is not positive definite");
    return r;
}

int32_t lu_apply_launch(ddg_problem *p, const double *r, const int *stop, cudaStream_t s) {
    k_lu_apply<<<p->K, LU_T, sizeof(double) * p->lu_kmax, s>>>(p->sub_ptr, p->sub_idx, p->lu_pos, p->lu_bw,
                                                             p->lu_off, p->lu_toff, p->lu_band, p->lu_bandT,
                                                             p->lu_tinv, r, p->s, p->corr, stop);
    DDG_LAUNCH_CHECK();
    return DDG_OK;
}

}  // namespace ddg
