// Overlapping decomposition on the device (Section II-A; Section IV-A):
//  * recursive coordinate bisection of the free nodes (the partitioner that
//    stands in for METIS): split along the longer bounding-box side, the lower
//    part takes floor(|S| floor(K/2) / K) nodes in the order (coordinate,
//    other coordinate, id).  Implemented with two presorted lists (by x and by
//    y) that every level splits by a stable partition, so no level re-sorts;
//  * overlap by adjacency layers of the A_ff graph (node -> sorted subdomain
//    sets, merged with the neighbours' sets once per layer);
//  * subdomain lists R_i (ascending free ids), partition-of-unity weights
//    1 / multiplicity (Nicolaides coarse space, Section II-A);
//  * the local DSS graphs of Section III-B: unknowns S_i then the halo (mesh
//    neighbours of S_i outside S_i, Dirichlet nodes included, ascending mesh
//    id); every mesh neighbour of an unknown is an in-neighbour, unknowns
//    point to unknown neighbours, halo nodes point to their unknown neighbours;
//  * A_0 = Z^T A Z (dense, FP64) and its inverse by pivot-free Gauss-Jordan
//    elimination (A_0 is SPD, so every pivot is positive).
#include "ddg_internal.cuh"

#include <algorithm>
#include <climits>

namespace ddg {

// ------------------------------------------------------------------ RCB
__global__ void k_seg_axis(const double *xy, const int *Lx, const int *Ly, const int *seg_start, const int *seg_len,
                           const int *seg_K, int nseg, int *seg_axis, int *seg_n1) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    int K = seg_K[s], st = seg_start[s], len = seg_len[s];
    if (K <= 1 || len == 0) {
        seg_axis[s] = -1;
        seg_n1[s] = len;
        return;
    }
    double ex = xy[2 * Lx[st + len - 1]] - xy[2 * Lx[st]];
    double ey = xy[2 * Ly[st + len - 1] + 1] - xy[2 * Ly[st] + 1];
    seg_axis[s] = (ex >= ey) ? 0 : 1;
    int K1 = K / 2;
    seg_n1[s] = (int)(((long long)len * K1) / K);
}

__device__ __forceinline__ int find_seg(const int *seg_start, int nseg, int p) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        int m = (lo + hi + 1) >> 1;
        if (seg_start[m] <= p) lo = m; else hi = m - 1;
    }
    return lo;
}

__global__ void k_mark_side(const int *Lx, const int *Ly, int nf, const int *seg_start, int nseg, const int *seg_axis,
                            const int *seg_n1, uint8_t *side) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nf) return;
    int s = find_seg(seg_start, nseg, p);
    int ax = seg_axis[s];
    if (ax < 0) return;
    int node = ax == 0 ? Lx[p] : Ly[p];
    side[node] = (p - seg_start[s] < seg_n1[s]) ? 0 : 1;
}

__global__ void k_left_flags(const int *L, int nf, const int *seg_start, int nseg, const int *seg_axis,
                             const uint8_t *side, int *flag) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nf) return;
    int s = find_seg(seg_start, nseg, p);
    flag[p] = (seg_axis[s] >= 0 && side[L[p]] == 0) ? 1 : 0;
}

__global__ void k_stable_split(const int *L, int *Lnew, int nf, const int *seg_start, int nseg, const int *seg_axis,
                               const int *seg_n1, const int *scan, const uint8_t *side) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nf) return;
    int s = find_seg(seg_start, nseg, p);
    int st = seg_start[s];
    int node = L[p];
    if (seg_axis[s] < 0) {
        Lnew[p] = node;
        return;
    }
    int left_before = scan[p] - scan[st];
    int pos = side[node] == 0 ? st + left_before : st + seg_n1[s] + (p - st - left_before);
    Lnew[pos] = node;
}

__global__ void k_part_from_segments(const int *L, int nf, const int *seg_start, int nseg, const int *seg_base,
                                     int *part) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nf) return;
    part[L[p]] = seg_base[find_seg(seg_start, nseg, p)];
}

static int32_t rcb(ddg_problem *p, int K) {
    ddg_ctx *c = p->ctx;
    cudaStream_t s = p->stream;
    const int nf = p->nf;
    Scratch sc(s);
    int *Lx, *Ly, *Ln, *flag, *scan;
    uint8_t *side;
    int *dseg;  // 6 arrays of K ints: start, len, K, base, axis, n1
    DDG_CU(sc.get(&Lx, nf));
    DDG_CU(sc.get(&Ly, nf));
    DDG_CU(sc.get(&Ln, nf));
    DDG_CU(sc.get(&flag, nf + 1));
    DDG_CU(sc.get(&scan, nf + 1));
    DDG_CU(sc.get(&side, nf));
    DDG_CU(sc.get(&dseg, 6LL * K));
    DDG_TRY(sort_points(c, p->xy_free, nf, 0, Lx, s));
    DDG_TRY(sort_points(c, p->xy_free, nf, 1, Ly, s));
    std::vector<int> st{0}, len{nf}, kk{K}, base{0};
    std::vector<int> axis(K), n1(K);
    int *d_st = dseg, *d_len = dseg + K, *d_K = dseg + 2 * K, *d_base = dseg + 3 * K, *d_ax = dseg + 4 * K,
        *d_n1 = dseg + 5 * K;
    for (int level = 0; level < 64; ++level) {
        bool active = false;
        for (int v : kk) active |= v > 1;
        if (!active) break;
        int ns = (int)st.size();
        DDG_CU(cudaMemcpyAsync(d_st, st.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
        DDG_CU(cudaMemcpyAsync(d_len, len.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
        DDG_CU(cudaMemcpyAsync(d_K, kk.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
        k_seg_axis<<<cdiv(ns, 128), 128, 0, s>>>(p->xy_free, Lx, Ly, d_st, d_len, d_K, ns, d_ax, d_n1);
        DDG_LAUNCH_CHECK();
        k_mark_side<<<cdiv(nf, 256), 256, 0, s>>>(Lx, Ly, nf, d_st, ns, d_ax, d_n1, side);
        DDG_LAUNCH_CHECK();
        for (int which = 0; which < 2; ++which) {
            int *L = which == 0 ? Lx : Ly;
            k_left_flags<<<cdiv(nf, 256), 256, 0, s>>>(L, nf, d_st, ns, d_ax, side, flag);
            DDG_LAUNCH_CHECK();
            DDG_CU(cudaMemsetAsync(flag + nf, 0, sizeof(int), s));
            DDG_TRY(scan_exclusive(c, flag, scan, nf + 1, nullptr, s));
            k_stable_split<<<cdiv(nf, 256), 256, 0, s>>>(L, Ln, nf, d_st, ns, d_ax, d_n1, scan, side);
            DDG_LAUNCH_CHECK();
            DDG_CU(cudaMemcpyAsync(L, Ln, sizeof(int) * nf, cudaMemcpyDeviceToDevice, s));
        }
        DDG_CU(cudaMemcpyAsync(axis.data(), d_ax, sizeof(int) * ns, cudaMemcpyDeviceToHost, s));
        DDG_CU(cudaMemcpyAsync(n1.data(), d_n1, sizeof(int) * ns, cudaMemcpyDeviceToHost, s));
        DDG_CU(cudaStreamSynchronize(s));
        std::vector<int> st2, len2, kk2, base2;
        for (int q = 0; q < ns; ++q) {
            if (axis[q] < 0) {
                st2.push_back(st[q]); len2.push_back(len[q]); kk2.push_back(kk[q]); base2.push_back(base[q]);
            } else {
                int K1 = kk[q] / 2;
                st2.push_back(st[q]); len2.push_back(n1[q]); kk2.push_back(K1); base2.push_back(base[q]);
                st2.push_back(st[q] + n1[q]); len2.push_back(len[q] - n1[q]); kk2.push_back(kk[q] - K1);
                base2.push_back(base[q] + K1);
            }
        }
        st.swap(st2); len.swap(len2); kk.swap(kk2); base.swap(base2);
    }
    int ns = (int)st.size();
    for (int q = 0; q < ns; ++q) {
        if (len[q] == 0) {
            set_error("recursive bisection produced an empty part: K exceeds the number of free nodes");
            return DDG_INVALID_ARG;
        }
    }
    DDG_CU(cudaMemcpyAsync(d_st, st.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
    DDG_CU(cudaMemcpyAsync(d_base, base.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
    k_part_from_segments<<<cdiv(nf, 256), 256, 0, s>>>(Lx, nf, d_st, ns, d_base, p->part);
    DDG_LAUNCH_CHECK();
    return DDG_OK;
}

// ------------------------------------------------------------------ overlap
__global__ void k_check_part(const int *part, int nf, int K, int *st, int *cnt) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int v = part[f];
    if (v < 0 || v >= K) {
        raise_status(st, ST_BAD_INPUT);
        return;
    }
    atomicAdd(&cnt[v], 1);
}

__global__ void k_mem_init(const int *part, int nf, int *mptr, int *midx) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f > nf) return;
    mptr[f] = f;
    if (f < nf) midx[f] = part[f];
}

constexpr int MEM_GATHER = 192;

// one overlap layer: new set of f = union of the sets of f and of its A_ff neighbours
__global__ void k_mem_layer(const int *rowptr, const int *col, const int *mptr, const int *midx, int nf, int pass,
                            int *cnt, const int *nptr, int *nidx, int *st) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int buf[MEM_GATHER];
    int m = 0;
    bool over = false;
    for (int e = rowptr[f]; e < rowptr[f + 1]; ++e) {
        int l = col[e];
        for (int q = mptr[l]; q < mptr[l + 1]; ++q) {
            if (m < MEM_GATHER) buf[m++] = midx[q]; else over = true;
        }
    }
    if (over) {
        raise_status(st, ST_TOO_LARGE);
        return;
    }
    insertion_sort(buf, m);
    int u = 0;
    int out = pass ? nptr[f] : 0;
    for (int k = 0; k < m; ++k) {
        if (k > 0 && buf[k] == buf[k - 1]) continue;
        if (pass) nidx[out + u] = buf[k];
        ++u;
    }
    if (!pass) {
        if (u > MAX_MEMBERSHIP) raise_status(st, ST_TOO_LARGE);
        cnt[f] = u;
    }
}

__global__ void k_pairs(const int *mptr, const int *midx, int nf, int *pnode, int *psub, int *mult,
                        double *inv_mult) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    for (int q = mptr[f]; q < mptr[f + 1]; ++q) {
        pnode[q] = f;
        psub[q] = midx[q];
    }
    const int m = mptr[f + 1] - mptr[f];
    mult[f] = m;
    inv_mult[f] = 1.0 / m;  // the partition-of-unity weight, divided once here
}

__global__ void k_sub_lists(const int *order, const int *pnode, const int *psub, int total, int *sub_idx,
                            int *inv_pos, int *sub_cnt) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= total) return;
    int src = order[q];
    sub_idx[q] = pnode[src];
    inv_pos[src] = q;
    atomicAdd(&sub_cnt[psub[src]], 1);
}

// ------------------------------------------------------------------ local graphs
constexpr int LG_T = 256;
constexpr int MAX_CAND = 4096;
constexpr int MAX_LOC = 6144;

__device__ __forceinline__ bool in_sub(const int *mptr, const int *midx, int f, int i) {
    for (int q = mptr[f]; q < mptr[f + 1]; ++q)
        if (midx[q] == i) return true;
    return false;
}

__device__ __forceinline__ int lower_bound_i(const int *a, int n, int v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int m = (lo + hi) >> 1;
        if (a[m] < v) lo = m + 1; else hi = m;
    }
    return lo;
}

// sorted unique halo (mesh ids) of subdomain i into sh; returns its size or -1 on overflow (all threads)
__device__ int build_halo(int i, const int *S, int k, const int *free_node, const int *aptr, const int *aidx,
                          const uint8_t *dir, const int *free_id, const int *mptr, const int *midx, int *sh,
                          int *sh_cnt) {
    if (threadIdx.x == 0) *sh_cnt = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        int a = free_node[S[t]];
        for (int e = aptr[a]; e < aptr[a + 1]; ++e) {
            int v = aidx[e];
            if (dir[v] || !in_sub(mptr, midx, free_id[v], i)) {
                int pos = atomicAdd(sh_cnt, 1);
                if (pos < MAX_CAND) sh[pos] = v;
            }
        }
    }
    __syncthreads();
    int cnt = *sh_cnt;
    if (cnt > MAX_CAND) return -1;
    int N = 1;
    while (N < cnt) N <<= 1;
    for (int q = cnt + threadIdx.x; q < N; q += blockDim.x) sh[q] = INT_MAX;
    __syncthreads();
    for (int kk = 2; kk <= N; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int q = threadIdx.x; q < N; q += blockDim.x) {
                int r = q ^ j;
                if (r > q) {
                    bool up = (q & kk) == 0;
                    int a = sh[q], b = sh[r];
                    if ((a > b) == up) { sh[q] = b; sh[r] = a; }
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        int u = 0;
        for (int q = 0; q < cnt; ++q)
            if (q == 0 || sh[q] != sh[q - 1]) sh[u++] = sh[q];
        *sh_cnt = u;
    }
    __syncthreads();
    return *sh_cnt;
}

__global__ void __launch_bounds__(LG_T) k_graph_count(const int *sub_ptr, const int *sub_idx, const int *free_node,
                                                      const int *aptr, const int *aidx, const uint8_t *dir,
                                                      const int *free_id, const int *mptr, const int *midx,
                                                      int *n_loc, int *n_edge, int *st) {
    __shared__ int sh[MAX_CAND];
    __shared__ int sh_cnt;
    __shared__ int sh_e;
    int i = blockIdx.x;
    const int *S = sub_idx + sub_ptr[i];
    int k = sub_ptr[i + 1] - sub_ptr[i];
    int nh = build_halo(i, S, k, free_node, aptr, aidx, dir, free_id, mptr, midx, sh, &sh_cnt);
    if (nh < 0 || k + nh > MAX_LOC) {
        if (threadIdx.x == 0) {
            raise_status(st, ST_TOO_LARGE);
            n_loc[i] = 0;
            n_edge[i] = 0;
        }
        return;
    }
    if (threadIdx.x == 0) sh_e = 0;
    __syncthreads();
    int e = 0;
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        int a = free_node[S[t]];
        e += aptr[a + 1] - aptr[a];
    }
    for (int h = threadIdx.x; h < nh; h += blockDim.x) {
        int v = sh[h];
        for (int q = aptr[v]; q < aptr[v + 1]; ++q) {
            int w = aidx[q];
            if (!dir[w] && in_sub(mptr, midx, free_id[w], i)) ++e;
        }
    }
    atomicAdd(&sh_e, e);
    __syncthreads();
    if (threadIdx.x == 0) {
        n_loc[i] = k + nh;
        n_edge[i] = sh_e;
    }
}

// in-place exclusive scan of a[0..n) by one block
__device__ void block_scan_excl(int *a, int n, int *sh_tmp /* >= 32 ints */) {
    int T = blockDim.x;
    int chunk = (n + T - 1) / T;
    int b0 = threadIdx.x * chunk, b1 = min(n, b0 + chunk);
    int s = 0;
    for (int q = b0; q < b1; ++q) s += a[q];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = s;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh_tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (T >> 5) ? sh_tmp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh_tmp[lane] = w;
    }
    __syncthreads();
    int run = x - s + (warp > 0 ? sh_tmp[warp - 1] : 0);
    for (int q = b0; q < b1; ++q) {
        int v = a[q];
        a[q] = run;
        run += v;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(LG_T) k_graph_fill(const int *sub_ptr, const int *sub_idx, const int *free_node,
                                                     const int *aptr, const int *aidx, const uint8_t *dir,
                                                     const int *free_id, const int *mptr, const int *midx,
                                                     const double *xy, double hbar, const int *loc_ptr,
                                                     const int *nbr_off, int *loc_nint, int *loc_node,
                                                     float2 *loc_xy, int *nbr_ptr, uint16_t *nbr) {
    __shared__ int sh[MAX_CAND];
    __shared__ int sh_cnt;
    __shared__ int cnt[MAX_LOC + 1];
    __shared__ int sh_tmp[32];
    __shared__ double red[32];
    int i = blockIdx.x;
    const int *S = sub_idx + sub_ptr[i];
    int k = sub_ptr[i + 1] - sub_ptr[i];
    int nh = build_halo(i, S, k, free_node, aptr, aidx, dir, free_id, mptr, midx, sh, &sh_cnt);
    int nl = loc_ptr[i + 1] - loc_ptr[i];
    if (nh < 0 || nl != k + nh) return;  // flagged by k_graph_count
    int lp = loc_ptr[i];
    if (threadIdx.x == 0) loc_nint[i] = k;
    // centre of the unknowns
    double sx = 0.0, sy = 0.0;
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        int a = free_node[S[t]];
        sx += xy[2 * a];
        sy += xy[2 * a + 1];
    }
    sx = block_sum(sx, red);
    if (threadIdx.x == 0) red[31] = sx;
    __syncthreads();
    sx = red[31];
    __syncthreads();
    sy = block_sum(sy, red);
    if (threadIdx.x == 0) red[31] = sy;
    __syncthreads();
    sy = red[31];
    double cx = sx / k, cy = sy / k;
    for (int q = threadIdx.x; q < nl; q += blockDim.x) {
        int v = q < k ? free_node[S[q]] : sh[q - k];
        loc_node[lp + q] = v;
        loc_xy[lp + q] = make_float2((float)((xy[2 * v] - cx) / hbar), (float)((xy[2 * v + 1] - cy) / hbar));
        int c;
        if (q < k) {
            c = aptr[v + 1] - aptr[v];
        } else {
            c = 0;
            for (int e = aptr[v]; e < aptr[v + 1]; ++e) {
                int w = aidx[e];
                if (!dir[w] && in_sub(mptr, midx, free_id[w], i)) ++c;
            }
        }
        cnt[q] = c;
    }
    if (threadIdx.x == 0) cnt[nl] = 0;
    __syncthreads();
    block_scan_excl(cnt, nl + 1, sh_tmp);
    int *np = nbr_ptr + lp + i;
    uint16_t *nb = nbr + nbr_off[i];
    for (int q = threadIdx.x; q <= nl; q += blockDim.x) np[q] = cnt[q];
    for (int q = threadIdx.x; q < nl; q += blockDim.x) {
        int v = q < k ? free_node[S[q]] : sh[q - k];
        int o = cnt[q];
        for (int e = aptr[v]; e < aptr[v + 1]; ++e) {
            int w = aidx[e];
            bool inner = !dir[w] && in_sub(mptr, midx, free_id[w], i);
            if (inner) {
                nb[o++] = (uint16_t)lower_bound_i(S, k, free_id[w]);
            } else if (q < k) {
                nb[o++] = (uint16_t)(k + lower_bound_i(sh, nh, w));
            }
        }
    }
}

// ------------------------------------------------------------------ coarse space
// A_0[a][b] = sum_{j in S_a} sum_{l in row j, b in sets(l)} A_jl / (m_j m_l), one CTA per row a:
// the CTA first collects the subdomains b that can appear (a bitmap over K), then
// one warp per b sums over S_a with a fixed lane assignment and a fixed shuffle tree.
constexpr int CO_T = 256;
constexpr int CO_MAX_NB = 256;

__global__ void __launch_bounds__(CO_T) k_coarse_rows(const int *sub_ptr, const int *sub_idx, const int *rowptr,
                                                      const int *col, const double *val, const int *mptr,
                                                      const int *midx, const int *mult, int K, double *A0,
                                                      int *st) {
    extern __shared__ unsigned int bits[];  // ceil(K / 32) words
    __shared__ int nb_list[CO_MAX_NB];
    __shared__ int nb_count;
    const int a = blockIdx.x;
    const int words = (K + 31) / 32;
    for (int q = threadIdx.x; q < words; q += CO_T) bits[q] = 0u;
    if (threadIdx.x == 0) nb_count = 0;
    __syncthreads();
    const int q0 = sub_ptr[a], q1 = sub_ptr[a + 1];
    for (int q = q0 + threadIdx.x; q < q1; q += CO_T) {
        int j = sub_idx[q];
        for (int e = rowptr[j]; e < rowptr[j + 1]; ++e) {
            int l = col[e];
            for (int r = mptr[l]; r < mptr[l + 1]; ++r) {
                int b = midx[r];
                atomicOr(&bits[b >> 5], 1u << (b & 31));
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int c = 0;
        for (int wd = 0; wd < words; ++wd) {
            unsigned int m = bits[wd];
            while (m) {
                int bit = __ffs(m) - 1;
                m &= m - 1;
                if (c < CO_MAX_NB) nb_list[c] = wd * 32 + bit;
                ++c;
            }
        }
        nb_count = c;
        if (c > CO_MAX_NB) raise_status(st, ST_TOO_LARGE);
    }
    __syncthreads();
    const int nbc = min(nb_count, CO_MAX_NB);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int u = warp; u < nbc; u += CO_T / 32) {
        const int b = nb_list[u];
        double acc = 0.0;
        for (int q = q0 + lane; q < q1; q += 32) {
            int j = sub_idx[q];
            double wa = 1.0 / mult[j];
            for (int e = rowptr[j]; e < rowptr[j + 1]; ++e) {
                int l = col[e];
                bool hit = false;
                for (int r = mptr[l]; r < mptr[l + 1]; ++r) hit |= midx[r] == b;
                if (hit) acc += wa * val[e] * (1.0 / mult[l]);
            }
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) A0[(long long)a * K + b] = acc;
    }
}

// Inverse of the SPD coarse matrix by blocked Gauss-Jordan elimination, in place, pivot blocks
// of GJB rows taken in order (no pivoting: every leading block of an SPD matrix and each Schur
// complement stay SPD).  Step k with the pivot block A_kk and P = A_kk^-1:
//   A_kj <- P A_kj,  A_ij <- A_ij - A_ik (P A_kj),  A_ik <- -A_ik P  (i, j != k),  A_kk <- P,
// the block form of the scalar sweep a_kj /= a_kk, a_ij -= a_ik a_kj, a_ik = -a_ik / a_kk,
// a_kk = 1 / a_kk; after the last step A holds A^-1.  Three launches per step: the pivot
// block's inverse (one CTA, scalar Gauss-Jordan in shared memory), the panel (P times row
// block k, and a copy of column block k), and the update of every element from the panel.
constexpr int GJB = 32;

__global__ void __launch_bounds__(GJB *GJB) k_bgj_pivot(const double *A, int K, int k0, int nb, double *P, int *st) {
    __shared__ double M[GJB][GJB + 1];
    __shared__ double prow[GJB], fcol[GJB], rpiv;
    const int i = threadIdx.y, j = threadIdx.x;
    M[i][j] = (i < nb && j < nb) ? A[(long long)(k0 + i) * K + k0 + j] : (i == j ? 1.0 : 0.0);
    __syncthreads();
    bool bad = false;
    for (int k = 0; k < nb; ++k) {
        if (i == 0 && j == 0) {
            const double piv = M[k][k];
            bad |= !(piv > 0.0);
            rpiv = 1.0 / piv;
        }
        __syncthreads();
        if (i == 0) prow[j] = (j == k ? 1.0 : M[k][j]) * rpiv;
        if (j == 0) fcol[i] = M[i][k];
        __syncthreads();
        M[i][j] = (i == k) ? prow[j] : ((j == k ? 0.0 : M[i][j]) - fcol[i] * prow[j]);
        __syncthreads();
    }
    P[i * GJB + j] = M[i][j];
    if (bad) raise_status(st, ST_BAD_INPUT);
}

// R = P A[k0 .. k0 + nb)[:] (nb x K, row-major), C = A[:][k0 .. k0 + nb) (K x GJB, row-major):
// 32 columns per CTA, a thread four rows of R in one column and one column's C entries
__global__ void __launch_bounds__(256) k_bgj_panel(const double *A, int K, int k0, int nb, const double *P,
                                                   double *R, double *C) {
    __shared__ double Ps[GJB][GJB + 1], As[GJB][GJB + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const int j = blockIdx.x * GJB + tx;
    for (int rr = ty; rr < GJB; rr += 8) {
        Ps[rr][tx] = P[rr * GJB + tx];
        As[rr][tx] = (rr < nb && j < K) ? A[(long long)(k0 + rr) * K + j] : 0.0;
    }
    __syncthreads();
    if (j < K)
        for (int r = ty; r < nb; r += 8) {
            double acc = 0.0;
#pragma unroll 8
            for (int m = 0; m < GJB; ++m) acc += Ps[r][m] * As[m][tx];
            R[(long long)r * K + j] = acc;
        }
    // column block k of row j (the rows of this CTA's columns, read along the row)
    for (int rr = ty; rr < GJB; rr += 8) {
        const int row = blockIdx.x * GJB + rr;
        if (row < K) C[(long long)row * GJB + tx] = tx < nb ? A[(long long)row * K + k0 + tx] : 0.0;
    }
}

// every element from the panel; tiles of 32 x 32, a thread four rows of one column
__global__ void __launch_bounds__(256) k_bgj_update(double *A, int K, int k0, int nb, const double *P,
                                                    const double *R, const double *C) {
    __shared__ double Cs[GJB][GJB + 1], Rs[GJB][GJB + 1], Ps[GJB][GJB + 1];
    const int i0 = blockIdx.y * GJB, j0 = blockIdx.x * GJB;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const bool col_k = j0 < k0 + nb && j0 + GJB > k0;        // the tile meets column block k
    for (int rr = ty; rr < GJB; rr += 8) {
        const int i = i0 + rr, j = j0 + tx;
        Cs[rr][tx] = i < K ? C[(long long)i * GJB + tx] : 0.0;
        Rs[rr][tx] = (rr < nb && j < K) ? R[(long long)rr * K + j] : 0.0;
        if (col_k) Ps[rr][tx] = P[rr * GJB + tx];
    }
    __syncthreads();
    const int j = j0 + tx;
    if (j >= K) return;
    const bool in_j = j >= k0 && j < k0 + nb;
    for (int rr = ty; rr < GJB; rr += 8) {
        const int i = i0 + rr;
        if (i >= K) break;
        const bool in_i = i >= k0 && i < k0 + nb;
        double v;
        if (in_i && in_j) {
            v = Ps[i - k0][j - k0];
        } else if (in_i) {
            v = Rs[i - k0][tx];
        } else if (in_j) {
            double acc = 0.0;
            for (int m = 0; m < nb; ++m) acc += Cs[rr][m] * Ps[m][j - k0];
            v = -acc;
        } else {
            double acc = 0.0;
            for (int m = 0; m < nb; ++m) acc += Cs[rr][m] * Rs[m][tx];
            v = A[(long long)i * K + j] - acc;
        }
        A[(long long)i * K + j] = v;
    }
}

int32_t coarse_build(ddg_problem *p) {
    ddg_ctx *c = p->ctx;
    cudaStream_t s = p->stream;
    const int K = p->K;
    DDG_TRY(dalloc(c, p->a_part, &p->A0, (size_t)K * K));
    DDG_TRY(dalloc(c, p->a_part, &p->A0inv, (size_t)K * K));
    DDG_CU(cudaMemsetAsync(p->A0, 0, sizeof(double) * K * K, s));
    size_t co_smem = sizeof(unsigned int) * ((K + 31) / 32);
    if (co_smem > 48 * 1024) {
        set_error("K too large for the coarse-matrix kernel");
        return DDG_TOO_LARGE;
    }
    k_coarse_rows<<<K, CO_T, co_smem, s>>>(p->sub_ptr, p->sub_idx, p->rowptr, p->col, p->val, p->mem_ptr,
                                           p->mem_idx, p->mult, K, p->A0, p->d_status);
    DDG_LAUNCH_CHECK();
    DDG_TRY(check_status(p, "coarse matrix"));
    DDG_CU(cudaMemcpyAsync(p->A0inv, p->A0, sizeof(double) * K * K, cudaMemcpyDeviceToDevice, s));
    Scratch sc(s);
    double *Pk, *Rk, *Ck;
    DDG_CU(sc.get(&Pk, GJB * GJB));
    DDG_CU(sc.get(&Rk, (size_t)GJB * K));
    DDG_CU(sc.get(&Ck, (size_t)GJB * K));
    const dim3 tiles(cdiv(K, GJB), cdiv(K, GJB));
    int steps = 0;
    for (int k0 = 0; k0 < K; k0 += GJB, ++steps) {
        const int nb = std::min(GJB, K - k0);
        k_bgj_pivot<<<1, dim3(GJB, GJB), 0, s>>>(p->A0inv, K, k0, nb, Pk, p->d_status);
        k_bgj_panel<<<cdiv(K, GJB), 256, 0, s>>>(p->A0inv, K, k0, nb, Pk, Rk, Ck);
        k_bgj_update<<<tiles, 256, 0, s>>>(p->A0inv, K, k0, nb, Pk, Rk, Ck);
    }
    DDG_LAUNCH_CHECK();
    DDG_LAUNCHES(3 * steps);
    DDG_CU(sc.drop(Pk));
    DDG_CU(sc.drop(Rk));
    DDG_CU(sc.drop(Ck));
    DDG_CU(cudaStreamSynchronize(s));
    int32_t r = check_status(p, "coarse inverse");
    if (r == DDG_INVALID_ARG) set_error("coarse matrix A_0 is not positive definite");
    return r;
}

// ------------------------------------------------------------------ driver
__global__ void k_neg(const int *in, int n, int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = -in[i];
}

__global__ void k_diff(const int *ptr, int n, int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ptr[i + 1] - ptr[i];
}

__global__ void k_iota_i(int *a, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = i;
}

int32_t partition_build(ddg_problem *p, int K, int delta, const int *part_host) {
    ddg_ctx *c = p->ctx;
    cudaStream_t s = p->stream;
    dfree_all(c, p->a_kry);
    dfree_all(c, p->a_pre);
    chunk_free(p);
    dfree_all(c, p->a_part);
    p->kind = DDG_NONE;
    p->K = 0;
    const int nf = p->nf;
    Scratch sc(s);
    DDG_TRY(dalloc(c, p->a_part, &p->part, nf));
    if (part_host) {
        DDG_CU(cudaMemcpyAsync(p->part, part_host, sizeof(int) * nf, cudaMemcpyHostToDevice, s));
    } else {
        DDG_TRY(rcb(p, K));
    }
    int *cnt;
    DDG_CU(sc.get(&cnt, std::max(nf, K) + 1));
    DDG_CU(cudaMemsetAsync(cnt, 0, sizeof(int) * K, s));
    k_check_part<<<cdiv(nf, 256), 256, 0, s>>>(p->part, nf, K, p->d_status, cnt);
    DDG_LAUNCH_CHECK();
    DDG_TRY(check_status(p, "partition"));
    {
        std::vector<int> h(K);
        DDG_CU(cudaMemcpyAsync(h.data(), cnt, sizeof(int) * K, cudaMemcpyDeviceToHost, s));
        DDG_CU(cudaStreamSynchronize(s));
        for (int i = 0; i < K; ++i)
            if (h[i] == 0) {
                set_error("part " + std::to_string(i) + " is empty");
                return DDG_INVALID_ARG;
            }
    }
    // membership sets, grown layer by layer
    int *mptr, *midx;
    DDG_CU(sc.get(&mptr, nf + 1));
    DDG_CU(sc.get(&midx, nf));
    k_mem_init<<<cdiv(nf + 1, 256), 256, 0, s>>>(p->part, nf, mptr, midx);
    DDG_LAUNCH_CHECK();
    int total = nf;
    for (int layer = 0; layer < delta; ++layer) {
        int *nptr, *nidx;
        DDG_CU(sc.get(&nptr, nf + 1));
        k_mem_layer<<<cdiv(nf, 128), 128, 0, s>>>(p->rowptr, p->col, mptr, midx, nf, 0, nptr, nullptr, nullptr,
                                                  p->d_status);
        DDG_LAUNCH_CHECK();
        DDG_TRY(check_status(p, "overlap"));
        DDG_CU(cudaMemsetAsync(nptr + nf, 0, sizeof(int), s));
        DDG_TRY(scan_exclusive(c, nptr, nptr, nf + 1, &total, s));
        DDG_CU(sc.get(&nidx, total));
        k_mem_layer<<<cdiv(nf, 128), 128, 0, s>>>(p->rowptr, p->col, mptr, midx, nf, 1, nullptr, nptr, nidx,
                                                  p->d_status);
        DDG_LAUNCH_CHECK();
        DDG_CU(sc.drop(mptr));
        DDG_CU(sc.drop(midx));
        mptr = nptr;
        midx = nidx;
    }
    DDG_TRY(dalloc(c, p->a_part, &p->mem_ptr, nf + 1));
    DDG_TRY(dalloc(c, p->a_part, &p->mem_idx, total));
    DDG_CU(cudaMemcpyAsync(p->mem_ptr, mptr, sizeof(int) * (nf + 1), cudaMemcpyDeviceToDevice, s));
    DDG_CU(cudaMemcpyAsync(p->mem_idx, midx, sizeof(int) * total, cudaMemcpyDeviceToDevice, s));
    DDG_CU(sc.drop(mptr));
    DDG_CU(sc.drop(midx));
    p->sum_k = total;

    // subdomain lists: pairs (node, sub) sorted by (sub, node)
    int *pnode, *psub, *order;
    DDG_CU(sc.get(&pnode, total));
    DDG_CU(sc.get(&psub, total));
    DDG_CU(sc.get(&order, total));
    DDG_TRY(dalloc(c, p->a_part, &p->mult, nf));
    DDG_TRY(dalloc(c, p->a_part, &p->inv_mult, nf));
    k_pairs<<<cdiv(nf, 256), 256, 0, s>>>(p->mem_ptr, p->mem_idx, nf, pnode, psub, p->mult, p->inv_mult);
    DDG_LAUNCH_CHECK();
    DDG_TRY(sort_pairs(c, psub, pnode, total, order, s));
    DDG_TRY(dalloc(c, p->a_part, &p->sub_idx, total));
    DDG_TRY(dalloc(c, p->a_part, &p->inv_pos, total));
    DDG_TRY(dalloc(c, p->a_part, &p->sub_ptr, K + 1));
    DDG_CU(cudaMemsetAsync(p->sub_ptr, 0, sizeof(int) * (K + 1), s));
    k_sub_lists<<<cdiv(total, 256), 256, 0, s>>>(order, pnode, psub, total, p->sub_idx, p->inv_pos, p->sub_ptr);
    DDG_LAUNCH_CHECK();
    DDG_TRY(scan_exclusive(c, p->sub_ptr, p->sub_ptr, K + 1, nullptr, s));
    DDG_CU(sc.drop(pnode));
    DDG_CU(sc.drop(psub));
    DDG_CU(sc.drop(order));
    p->K = K;
    p->delta = delta;

    // local graphs
    int *n_loc, *n_edge;
    DDG_CU(sc.get(&n_loc, K + 1));
    DDG_CU(sc.get(&n_edge, K + 1));
    k_graph_count<<<K, LG_T, 0, s>>>(p->sub_ptr, p->sub_idx, p->free_node, p->adj_ptr, p->adj_idx, p->dir,
                                      p->free_id, p->mem_ptr, p->mem_idx, n_loc, n_edge, p->d_status);
    DDG_LAUNCH_CHECK();
    DDG_TRY(check_status(p, "local graphs"));
    DDG_TRY(dalloc(c, p->a_part, &p->loc_ptr, K + 1));
    DDG_TRY(dalloc(c, p->a_part, &p->nbr_off, K + 1));
    DDG_TRY(dalloc(c, p->a_part, &p->loc_nint, K));
    {
        std::vector<int> h(K), he(K);
        DDG_CU(cudaMemcpyAsync(h.data(), n_loc, sizeof(int) * K, cudaMemcpyDeviceToHost, s));
        DDG_CU(cudaMemcpyAsync(he.data(), n_edge, sizeof(int) * K, cudaMemcpyDeviceToHost, s));
        DDG_CU(cudaStreamSynchronize(s));
        p->max_loc = *std::max_element(h.begin(), h.end());
        p->max_edges = *std::max_element(he.begin(), he.end());
    }
    DDG_CU(cudaMemsetAsync(n_loc + K, 0, sizeof(int), s));
    DDG_CU(cudaMemsetAsync(n_edge + K, 0, sizeof(int), s));
    int sum_loc = 0, sum_edge = 0;
    DDG_TRY(scan_exclusive(c, n_loc, p->loc_ptr, K + 1, &sum_loc, s));
    DDG_TRY(scan_exclusive(c, n_edge, p->nbr_off, K + 1, &sum_edge, s));
    p->sum_loc = sum_loc;
    p->sum_edges = sum_edge;
    DDG_TRY(dalloc(c, p->a_part, &p->loc_node, sum_loc));
    DDG_TRY(dalloc(c, p->a_part, &p->loc_xy, sum_loc));
    DDG_TRY(dalloc(c, p->a_part, &p->nbr_ptr, (size_t)sum_loc + K));
    DDG_TRY(dalloc(c, p->a_part, &p->nbr, sum_edge));
    k_graph_fill<<<K, LG_T, 0, s>>>(p->sub_ptr, p->sub_idx, p->free_node, p->adj_ptr, p->adj_idx, p->dir,
                                     p->free_id, p->mem_ptr, p->mem_idx, p->xy, p->hbar, p->loc_ptr, p->nbr_off,
                                     p->loc_nint, p->loc_node, p->loc_xy, p->nbr_ptr, p->nbr);
    DDG_LAUNCH_CHECK();
    // largest graphs first (the block scheduler then hands them out greedily)
    int *neg, *ids;
    DDG_CU(sc.get(&neg, K));
    DDG_CU(sc.get(&ids, K));
    DDG_TRY(dalloc(c, p->a_part, &p->lpt_order, K));
    k_diff<<<cdiv(K, 256), 256, 0, s>>>(p->loc_ptr, K, neg);
    k_neg<<<cdiv(K, 256), 256, 0, s>>>(neg, K, neg);
    k_iota_i<<<cdiv(K, 256), 256, 0, s>>>(ids, K);
    DDG_LAUNCHES(3);
    DDG_TRY(sort_pairs(c, neg, ids, K, p->lpt_order, s));
    DDG_CU(sc.drop(neg));
    DDG_CU(sc.drop(ids));
    DDG_CU(sc.drop(n_loc));
    DDG_CU(sc.drop(n_edge));
    DDG_CU(sc.drop(cnt));
    DDG_TRY(check_status(p, "local graphs"));
    return coarse_build(p);
}

}  // namespace ddg
