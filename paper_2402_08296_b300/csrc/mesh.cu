// Mesh topology and P1 Galerkin assembly (Section II, Eqs. 1-2), all on the device.
//
// Topology: node -> incident triangles (ascending), node -> mesh neighbours
// (ascending), boundary edges (edges in one triangle) give the default
// Dirichlet nodes, h_bar = mean edge length.
// Assembly is node-centric: one thread per free node walks its triangles in
// ascending order and accumulates its matrix row and its load, so the result
// is deterministic and A is bitwise symmetric (both (i,j) and (j,i) sum the
// same products in the same order).  Products and sums use explicitly rounded
// FP64 operations (no contraction), in the order the formulas are written:
//   K_T[i][k] = (b_i b_k + c_i c_k) / (4 |T|),  |T| = |b_0 c_1 - b_1 c_0| / 2,
//   int_T f lambda_i = |T| (f_i/30 - (f_j+f_l)/60 + 2 (f_ij+f_il)/15 + f_jl/15)
// (exact for quadratic f through its P2 interpolant), or |T|/12 (f_i + sum f)
// for nodal f (consistent mass).  Dirichlet data are eliminated: b_f -= A_fD g_D.
#include "ddg_internal.cuh"

namespace ddg {

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }

__global__ void k_tri_count(const double *xy, const int *tri, int n, int t, int *cnt, int *st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= t) return;
    int v0 = tri[3 * i], v1 = tri[3 * i + 1], v2 = tri[3 * i + 2];
    if (v0 < 0 || v1 < 0 || v2 < 0 || v0 >= n || v1 >= n || v2 >= n || v0 == v1 || v1 == v2 || v0 == v2) {
        raise_status(st, ST_BAD_MESH);
        return;
    }
    double ax = xy[2 * v0], ay = xy[2 * v0 + 1];
    double o = (xy[2 * v1] - ax) * (xy[2 * v2 + 1] - ay) - (xy[2 * v1 + 1] - ay) * (xy[2 * v2] - ax);
    if (!(o > 0.0)) raise_status(st, ST_BAD_MESH);
    atomicAdd(&cnt[v0], 1);
    atomicAdd(&cnt[v1], 1);
    atomicAdd(&cnt[v2], 1);
}

__global__ void k_tri_fill(const int *tri, int t, const int *ptr, int *fill, int *idx) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= t) return;
    for (int k = 0; k < 3; ++k) {
        int v = tri[3 * i + k];
        int slot = atomicAdd(&fill[v], 1);
        idx[ptr[v] + slot] = i;
    }
}

__global__ void k_sort_node_tris(const int *ptr, int *idx, int n, int *st) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    int b = ptr[a], m = ptr[a + 1] - b;
    if (m > MAX_NODE_TRI) {
        raise_status(st, ST_BAD_MESH);
        return;
    }
    int loc[MAX_NODE_TRI];
    for (int k = 0; k < m; ++k) loc[k] = idx[b + k];
    insertion_sort(loc, m);
    for (int k = 0; k < m; ++k) idx[b + k] = loc[k];
}

// pass 0: deg[a] and boundary flag; pass 1: neighbour lists
__global__ void k_node_nbr(const int *tri, const int *tptr, const int *tidx, int n, int pass, int *deg,
                           uint8_t *bnd, const int *aptr, int *aidx, int *st) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    int b0 = tptr[a], m = tptr[a + 1] - b0;
    if (m > MAX_NODE_TRI) return;  // flagged by k_sort_node_tris
    int o[2 * MAX_NODE_TRI];
    int cnt = 0;
    for (int k = 0; k < m; ++k) {
        int t = tidx[b0 + k];
        for (int q = 0; q < 3; ++q) {
            int v = tri[3 * t + q];
            if (v != a) o[cnt++] = v;
        }
    }
    insertion_sort(o, cnt);
    int u = 0;
    bool boundary = false;
    int out = pass ? aptr[a] : 0;
    for (int k = 0; k < cnt;) {
        int v = o[k], mult = 0;
        while (k < cnt && o[k] == v) { ++mult; ++k; }
        if (mult == 1) boundary = true;
        if (pass) aidx[out + u] = v;
        ++u;
    }
    if (!pass) {
        if (u > MAX_NODE_NBR) raise_status(st, ST_BAD_MESH);
        deg[a] = u;
        bnd[a] = boundary ? 1 : 0;
    }
}

__global__ void k_edge_len(const double *xy, const int *aptr, const int *aidx, int n, double *len) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    double s = 0.0;
    for (int k = aptr[a]; k < aptr[a + 1]; ++k) {
        int b = aidx[k];
        if (b > a) {
            double dx = xy[2 * b] - xy[2 * a], dy = xy[2 * b + 1] - xy[2 * a + 1];
            s += sqrt(dx * dx + dy * dy);
        }
    }
    len[a] = s;
}

__global__ void k_not_dir(const uint8_t *dir, int n, int *flag) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < n) flag[a] = dir[a] ? 0 : 1;
}

__global__ void k_free_ids(const uint8_t *dir, const double *xy, int n, int *free_id, int *free_node,
                           double *xy_free) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    if (dir[a]) {
        free_id[a] = -1;
    } else {
        int f = free_id[a];
        free_node[f] = a;
        xy_free[2 * f] = xy[2 * a];
        xy_free[2 * f + 1] = xy[2 * a + 1];
    }
}

int32_t mesh_build(ddg_problem *p, const uint8_t *dirichlet_host) {
    ddg_ctx *c = p->ctx;
    cudaStream_t s = p->stream;
    const int n = p->n, t = p->t;
    Scratch sc(s);
    int *cnt = nullptr, *fill = nullptr, *deg = nullptr;
    uint8_t *bnd = nullptr;
    DDG_CU(sc.get(&cnt, n + 1));
    DDG_CU(sc.get(&fill, n + 1));
    DDG_CU(sc.get(&deg, n + 1));
    DDG_CU(sc.get(&bnd, n));
    DDG_CU(cudaMemsetAsync(cnt, 0, sizeof(int) * (n + 1), s));
    DDG_CU(cudaMemsetAsync(fill, 0, sizeof(int) * (n + 1), s));

    k_tri_count<<<cdiv(t, 256), 256, 0, s>>>(p->xy, p->tri, n, t, cnt, p->d_status);
    DDG_LAUNCH_CHECK();
    DDG_TRY(check_status(p, "mesh upload"));
    DDG_TRY(dalloc(c, p->a_mesh, &p->ntri_ptr, n + 1));
    DDG_TRY(dalloc(c, p->a_mesh, &p->ntri_idx, 3LL * t));
    DDG_TRY(scan_exclusive(c, cnt, p->ntri_ptr, n + 1, nullptr, s));
    k_tri_fill<<<cdiv(t, 256), 256, 0, s>>>(p->tri, t, p->ntri_ptr, fill, p->ntri_idx);
    DDG_LAUNCH_CHECK();
    k_sort_node_tris<<<cdiv(n, 128), 128, 0, s>>>(p->ntri_ptr, p->ntri_idx, n, p->d_status);
    DDG_LAUNCH_CHECK();
    k_node_nbr<<<cdiv(n, 128), 128, 0, s>>>(p->tri, p->ntri_ptr, p->ntri_idx, n, 0, deg, bnd, nullptr, nullptr,
                                            p->d_status);
    DDG_LAUNCH_CHECK();
    DDG_TRY(check_status(p, "mesh upload"));
    DDG_CU(cudaMemsetAsync(deg + n, 0, sizeof(int), s));
    DDG_TRY(dalloc(c, p->a_mesh, &p->adj_ptr, n + 1));
    int total = 0;
    DDG_TRY(scan_exclusive(c, deg, p->adj_ptr, n + 1, &total, s));
    p->n_edges = total / 2;
    DDG_TRY(dalloc(c, p->a_mesh, &p->adj_idx, total));
    k_node_nbr<<<cdiv(n, 128), 128, 0, s>>>(p->tri, p->ntri_ptr, p->ntri_idx, n, 1, nullptr, nullptr, p->adj_ptr,
                                            p->adj_idx, p->d_status);
    DDG_LAUNCH_CHECK();

    DDG_TRY(dalloc(c, p->a_mesh, &p->dir, n));
    if (dirichlet_host) {
        DDG_CU(cudaMemcpyAsync(p->dir, dirichlet_host, n, cudaMemcpyHostToDevice, s));
    } else {
        DDG_CU(cudaMemcpyAsync(p->dir, bnd, n, cudaMemcpyDeviceToDevice, s));
    }

    // h_bar
    double *len = nullptr, *sum = nullptr;
    DDG_CU(sc.get(&len, n));
    DDG_CU(sc.get(&sum, 1));
    k_edge_len<<<cdiv(n, 256), 256, 0, s>>>(p->xy, p->adj_ptr, p->adj_idx, n, len);
    DDG_LAUNCH_CHECK();
    DDG_TRY(reduce_sum(c, len, n, sum, s));
    double hsum = 0.0;
    DDG_CU(cudaMemcpyAsync(&hsum, sum, sizeof(double), cudaMemcpyDeviceToHost, s));

    // free numbering
    DDG_TRY(dalloc(c, p->a_mesh, &p->free_id, n + 1));
    k_not_dir<<<cdiv(n, 256), 256, 0, s>>>(p->dir, n, p->free_id);
    DDG_LAUNCH_CHECK();
    int nf = 0;
    DDG_TRY(scan_exclusive(c, p->free_id, p->free_id, n, &nf, s));
    p->nf = nf;
    p->hbar = p->n_edges > 0 ? hsum / p->n_edges : 1.0;
    if (nf == 0) {
        set_error("mesh has no free node");
        return DDG_INVALID_ARG;
    }
    DDG_TRY(dalloc(c, p->a_mesh, &p->free_node, nf));
    DDG_TRY(dalloc(c, p->a_mesh, &p->xy_free, 2LL * nf));
    k_free_ids<<<cdiv(n, 256), 256, 0, s>>>(p->dir, p->xy, n, p->free_id, p->free_node, p->xy_free);
    DDG_LAUNCH_CHECK();

    DDG_CU(cudaStreamSynchronize(s));
    return check_status(p, "mesh upload");
}

// ------------------------------------------------------------------ assembly
struct Poly {
    double r[9];
};

__device__ __forceinline__ double poly_f(const Poly &q, double x, double y) {
    double xm = sub(x, 1.0);
    return add(add(mul(q.r[0], mul(xm, xm)), mul(q.r[1], mul(y, y))), q.r[2]);
}

__device__ __forceinline__ double poly_g(const Poly &q, double x, double y) {
    double v = add(mul(q.r[3], mul(x, x)), mul(q.r[4], mul(y, y)));
    v = add(v, mul(mul(q.r[5], x), y));
    v = add(v, mul(q.r[6], x));
    v = add(v, mul(q.r[7], y));
    return add(v, q.r[8]);
}

__global__ void k_dirichlet_values(const double *xy, const uint8_t *dir, int n, Poly q, const double *g_nodal,
                                   double *g) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    double v = 0.0;
    if (dir[a]) v = g_nodal ? g_nodal[a] : poly_g(q, xy[2 * a], xy[2 * a + 1]);
    g[a] = v;
}

__global__ void k_row_count(const int *free_node, const int *aptr, const int *aidx, const uint8_t *dir, int nf,
                            int *cnt) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int a = free_node[f];
    int c = 1;
    for (int k = aptr[a]; k < aptr[a + 1]; ++k) c += dir[aidx[k]] ? 0 : 1;
    cnt[f] = c;
}

__global__ void k_assemble(const double *xy, const int *tri, const int *tptr, const int *tidx, const int *aptr,
                           const int *aidx, const uint8_t *dir, const int *free_id, const int *free_node,
                           const double *g, int nf, Poly q, const double *f_nodal, const int *rowptr, int *col,
                           double *val, double *bvec) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int a = free_node[f];
    // row entries: a and its neighbours, ascending mesh id
    int ids[MAX_NODE_NBR + 1];
    double acc[MAX_NODE_NBR + 1];
    int m = 0;
    bool placed = false;
    for (int k = aptr[a]; k < aptr[a + 1]; ++k) {
        int v = aidx[k];
        if (!placed && a < v) { ids[m++] = a; placed = true; }
        ids[m++] = v;
    }
    if (!placed) ids[m++] = a;
    for (int k = 0; k < m; ++k) acc[k] = 0.0;
    double bacc = 0.0;
    for (int k = tptr[a]; k < tptr[a + 1]; ++k) {
        int t = tidx[k];
        int v[3];
        double x[3], y[3];
        int i = 0;
        for (int q3 = 0; q3 < 3; ++q3) {
            v[q3] = tri[3 * t + q3];
            x[q3] = xy[2 * v[q3]];
            y[q3] = xy[2 * v[q3] + 1];
            if (v[q3] == a) i = q3;
        }
        double bb[3] = {sub(y[1], y[2]), sub(y[2], y[0]), sub(y[0], y[1])};
        double cc[3] = {sub(x[2], x[1]), sub(x[0], x[2]), sub(x[1], x[0])};
        double area = mul(0.5, fabs(sub(mul(bb[0], cc[1]), mul(bb[1], cc[0]))));
        double den = mul(4.0, area);
        for (int k2 = 0; k2 < 3; ++k2) {
            double kik = add(mul(bb[i], bb[k2]), mul(cc[i], cc[k2])) / den;
            int pos = 0;
            while (ids[pos] != v[k2]) ++pos;
            acc[pos] = add(acc[pos], kik);
        }
        int j = (i + 1) % 3, l = (i + 2) % 3;
        double load;
        if (f_nodal) {
            double S = add(add(f_nodal[v[0]], f_nodal[v[1]]), f_nodal[v[2]]);
            load = mul(area / 12.0, add(f_nodal[v[i]], S));
        } else {
            double fi = poly_f(q, x[i], y[i]), fj = poly_f(q, x[j], y[j]), fl = poly_f(q, x[l], y[l]);
            double fij = poly_f(q, mul(0.5, add(x[i], x[j])), mul(0.5, add(y[i], y[j])));
            double fil = poly_f(q, mul(0.5, add(x[i], x[l])), mul(0.5, add(y[i], y[l])));
            double fjl = poly_f(q, mul(0.5, add(x[j], x[l])), mul(0.5, add(y[j], y[l])));
            double e = sub(fi / 30.0, add(fj, fl) / 60.0);
            e = add(e, mul(2.0, add(fij, fil)) / 15.0);
            e = add(e, fjl / 15.0);
            load = mul(area, e);
        }
        bacc = add(bacc, load);
    }
    int out = rowptr[f];
    double lift = 0.0;
    for (int k = 0; k < m; ++k) {
        int v = ids[k];
        if (dir[v]) {
            lift = add(lift, mul(acc[k], g[v]));
        } else {
            col[out] = free_id[v];
            val[out] = acc[k];
            ++out;
        }
    }
    bvec[f] = sub(bacc, lift);
}

int32_t assemble(ddg_problem *p, const double *r9, const double *f_nodal_host, const double *g_nodal_host) {
    ddg_ctx *c = p->ctx;
    cudaStream_t s = p->stream;
    dfree_all(c, p->a_kry);
    dfree_all(c, p->a_pre);
    chunk_free(p);
    dfree_all(c, p->a_part);
    dfree_all(c, p->a_matrix);
    p->assembled = false;
    p->K = 0;
    p->kind = DDG_NONE;
    const int n = p->n, nf = p->nf;
    Poly q{};
    if (r9) for (int k = 0; k < 9; ++k) q.r[k] = r9[k];
    Scratch sc(s);
    double *fn = nullptr, *gn = nullptr;
    if (f_nodal_host) {
        DDG_CU(sc.get(&fn, n));
        DDG_CU(sc.get(&gn, n));
        DDG_CU(cudaMemcpyAsync(fn, f_nodal_host, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        DDG_CU(cudaMemcpyAsync(gn, g_nodal_host, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    }
    DDG_TRY(dalloc(c, p->a_matrix, &p->g, n));
    k_dirichlet_values<<<cdiv(n, 256), 256, 0, s>>>(p->xy, p->dir, n, q, gn, p->g);
    DDG_LAUNCH_CHECK();
    DDG_TRY(dalloc(c, p->a_matrix, &p->rowptr, nf + 1));
    k_row_count<<<cdiv(nf, 256), 256, 0, s>>>(p->free_node, p->adj_ptr, p->adj_idx, p->dir, nf, p->rowptr);
    DDG_LAUNCH_CHECK();
    DDG_CU(cudaMemsetAsync(p->rowptr + nf, 0, sizeof(int), s));
    int nnz = 0;
    DDG_TRY(scan_exclusive(c, p->rowptr, p->rowptr, nf + 1, &nnz, s));
    p->nnz = nnz;
    DDG_TRY(dalloc(c, p->a_matrix, &p->col, nnz));
    DDG_TRY(dalloc(c, p->a_matrix, &p->val, nnz));
    DDG_TRY(dalloc(c, p->a_matrix, &p->b, nf));
    k_assemble<<<cdiv(nf, 128), 128, 0, s>>>(p->xy, p->tri, p->ntri_ptr, p->ntri_idx, p->adj_ptr, p->adj_idx,
                                             p->dir, p->free_id, p->free_node, p->g, nf, q, fn, p->rowptr,
                                             p->col, p->val, p->b);
    DDG_LAUNCH_CHECK();
    DDG_TRY(sell_build(p));
    DDG_CU(cudaStreamSynchronize(s));
    p->assembled = true;
    return check_status(p, "assemble");
}

}  // namespace ddg
