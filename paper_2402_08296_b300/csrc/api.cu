// The C ABI of libddg (declared in include/ddg.h): argument checks, object
// lifetime and stage ordering.  Every computational step runs in the kernels
// of the other translation units.
#include "ddg_internal.cuh"

#include <cstdlib>

#include <algorithm>
#include <cstring>


using namespace ddg;

#define API_BEGIN clear_error()
#define REQUIRE(cond, msg)              \
    do {                                \
        if (!(cond)) {                  \
            set_error(msg);             \
            return DDG_INVALID_ARG;     \
        }                               \
    } while (0)

static int32_t use_device(ddg_ctx *c) {
    DDG_CU(cudaSetDevice(c->device));
    return DDG_OK;
}

namespace ddg {

int32_t problem_create(ddg_ctx *c, int n_nodes, const double *xy, int n_tri, const int *tri, const uint8_t *dirichlet,
                       cudaStream_t stream, bool own_stream, ddg_problem **out) {
    ddg_problem *p = new ddg_problem();
    p->ctx = c;
    p->stream = stream;
    p->own_stream = own_stream;
    p->n = n_nodes;
    p->t = n_tri;
    for (ddg::Allocs *a : {&p->a_mesh, &p->a_matrix, &p->a_part, &p->a_pre, &p->a_kry, &p->a_hist, &p->chunk.allocs}) {
        a->stream = stream;
        a->use_stream = true;
    }
    int32_t st = DDG_OK;
    do {
        if ((st = dalloc(c, p->a_mesh, &p->d_status, 1)) != DDG_OK) break;
        if ((st = dalloc(c, p->a_mesh, &p->xy, 2LL * n_nodes)) != DDG_OK) break;
        if ((st = dalloc(c, p->a_mesh, &p->tri, 3LL * n_tri)) != DDG_OK) break;
        cudaMemsetAsync(p->d_status, 0, sizeof(int), p->stream);
        cudaMemcpyAsync(p->xy, xy, sizeof(double) * 2 * n_nodes, cudaMemcpyHostToDevice, p->stream);
        cudaMemcpyAsync(p->tri, tri, sizeof(int) * 3 * n_tri, cudaMemcpyHostToDevice, p->stream);
        st = mesh_build(p, dirichlet);
    } while (0);
    if (st != DDG_OK) {
        std::string msg = last_error_cstr();
        ddg_problem_destroy(p);
        set_error(msg);
        return st;
    }
    *out = p;
    return DDG_OK;
}

}  // namespace ddg

extern "C" {

const char *ddg_last_error(void) { return last_error_cstr(); }

int32_t ddg_create(int32_t device, size_t hbm_budget_bytes, ddg_ctx **out) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(out, "out is NULL");
        int count = 0;
        DDG_CU(cudaGetDeviceCount(&count));
        REQUIRE(device >= 0 && device < count, "no such CUDA device");
        DDG_CU(cudaSetDevice(device));
        ddg_ctx *c = new ddg_ctx();
        c->device = device;
        c->budget = hbm_budget_bytes;
        c->pdl = getenv("DDG_NO_PDL") == nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            set_error(std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
            return DDG_CUDA_ERROR;
        }
        *out = c;
        return DDG_OK;
    });
}

int32_t ddg_destroy(ddg_ctx *c) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        if (!c) return DDG_OK;
        server_stop(c);
        cudaSetDevice(c->device);
        cudaStreamSynchronize(c->stream);
        cudaStreamDestroy(c->stream);
        delete c;
        return DDG_OK;
    });
}

int32_t ddg_memory_in_use(ddg_ctx *c, size_t *bytes) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(c && bytes, "NULL argument");
        *bytes = c->in_use.load();
        return DDG_OK;
    });
}

int32_t ddg_get_stream(ddg_ctx *c, ddg_stream *out) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(c && out, "NULL argument");
        *out = (ddg_stream)c->stream;
        return DDG_OK;
    });
}

int32_t ddg_launch_count(uint64_t *out) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(out, "NULL argument");
        *out = (uint64_t)launch_count();
        return DDG_OK;
    });
}

// ------------------------------------------------------------------ mesh
int32_t ddg_mesh_upload(ddg_ctx *c, int32_t n_nodes, const double *xy, int32_t n_tri, const int32_t *tri,
                        const uint8_t *dirichlet, ddg_problem **out) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(c && xy && tri && out, "NULL argument");
        REQUIRE(n_nodes >= 3 && n_tri >= 1, "mesh needs at least one triangle");
        DDG_TRY(use_device(c));
        return problem_create(c, n_nodes, xy, n_tri, tri, dirichlet, c->stream, false, out);
    });
}

int32_t ddg_problem_destroy(ddg_problem *p) {
    return api_guard([&]() -> int32_t {
        if (!p) return DDG_OK;
        ddg_ctx *c = p->ctx;
        cudaSetDevice(c->device);
        cudaStreamSynchronize(p->stream);
        dfree_all(c, p->a_kry);
        dfree_all(c, p->a_hist);
        dfree_all(c, p->a_pre);
        chunk_free(p);
        dfree_all(c, p->a_part);
        dfree_all(c, p->a_matrix);
        dfree_all(c, p->a_mesh);
        if (p->hflag_pinned) cudaFreeHost(p->hflag_pinned);
        cudaStreamSynchronize(p->stream);
        if (p->own_stream) cudaStreamDestroy(p->stream);
        delete p;
        return DDG_OK;
    });
}

int32_t ddg_assemble_poly(ddg_problem *p, const double r[9]) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && r, "NULL argument");
        DDG_TRY(use_device(p->ctx));
        return assemble(p, r, nullptr, nullptr);
    });
}

int32_t ddg_assemble_nodal(ddg_problem *p, const double *f, const double *g) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && f && g, "NULL argument");
        DDG_TRY(use_device(p->ctx));
        return assemble(p, nullptr, f, g);
    });
}

int32_t ddg_problem_info(ddg_problem *p, int64_t info[10]) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && info, "NULL argument");
        for (int k = 0; k < 10; ++k) info[k] = -1;
        info[0] = p->n;
        info[1] = p->t;
        info[2] = p->nf;
        if (p->assembled) info[3] = p->nnz;
        if (p->K > 0) {
            info[4] = p->K;
            info[5] = p->sum_k;
            info[6] = p->sum_loc;
            info[7] = p->sum_edges;
            info[8] = p->max_loc;
        }
        std::memcpy(&info[9], &p->hbar, sizeof(double));
        return DDG_OK;
    });
}

int32_t ddg_matrix_download(ddg_problem *p, int32_t *rowptr, int32_t *col, double *val, double *b) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && p->assembled, "problem not assembled");
        DDG_TRY(use_device(p->ctx));
        cudaStream_t s = p->stream;
        if (rowptr) DDG_CU(cudaMemcpyAsync(rowptr, p->rowptr, sizeof(int) * (p->nf + 1), cudaMemcpyDeviceToHost, s));
        if (col) DDG_CU(cudaMemcpyAsync(col, p->col, sizeof(int) * p->nnz, cudaMemcpyDeviceToHost, s));
        if (val) DDG_CU(cudaMemcpyAsync(val, p->val, sizeof(double) * p->nnz, cudaMemcpyDeviceToHost, s));
        if (b) DDG_CU(cudaMemcpyAsync(b, p->b, sizeof(double) * p->nf, cudaMemcpyDeviceToHost, s));
        DDG_CU(cudaStreamSynchronize(s));
        return DDG_OK;
    });
}

// ------------------------------------------------------------------ decomposition
int32_t ddg_partition(ddg_problem *p, int32_t K, int32_t overlap_layers, const int32_t *part_or_null) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && p->assembled, "problem not assembled");
        REQUIRE(K >= 1 && K <= p->nf, "K must be in [1, n_free]");
        REQUIRE(overlap_layers >= 0 && overlap_layers <= 16, "overlap_layers must be in [0, 16]");
        DDG_TRY(use_device(p->ctx));
        return partition_build(p, K, overlap_layers, part_or_null);
    });
}

int32_t ddg_partition_download(ddg_problem *p, int32_t *part, int32_t *sub_ptr, int32_t *sub_idx, int32_t *mult) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && p->K > 0, "no partition");
        DDG_TRY(use_device(p->ctx));
        cudaStream_t s = p->stream;
        if (part) DDG_CU(cudaMemcpyAsync(part, p->part, sizeof(int) * p->nf, cudaMemcpyDeviceToHost, s));
        if (sub_ptr) DDG_CU(cudaMemcpyAsync(sub_ptr, p->sub_ptr, sizeof(int) * (p->K + 1), cudaMemcpyDeviceToHost, s));
        if (sub_idx) DDG_CU(cudaMemcpyAsync(sub_idx, p->sub_idx, sizeof(int) * p->sum_k, cudaMemcpyDeviceToHost, s));
        if (mult) DDG_CU(cudaMemcpyAsync(mult, p->mult, sizeof(int) * p->nf, cudaMemcpyDeviceToHost, s));
        DDG_CU(cudaStreamSynchronize(s));
        return DDG_OK;
    });
}

int32_t ddg_graph_download(ddg_problem *p, int32_t *loc_ptr, int32_t *n_int, int32_t *loc_node, int32_t *nbr_ptr,
                           int32_t *nbr) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && p->K > 0, "no partition");
        DDG_TRY(use_device(p->ctx));
        cudaStream_t s = p->stream;
        if (loc_ptr) DDG_CU(cudaMemcpyAsync(loc_ptr, p->loc_ptr, sizeof(int) * (p->K + 1), cudaMemcpyDeviceToHost, s));
        if (n_int) DDG_CU(cudaMemcpyAsync(n_int, p->loc_nint, sizeof(int) * p->K, cudaMemcpyDeviceToHost, s));
        if (loc_node) DDG_CU(cudaMemcpyAsync(loc_node, p->loc_node, sizeof(int) * p->sum_loc, cudaMemcpyDeviceToHost, s));
        if (nbr_ptr)
            DDG_CU(cudaMemcpyAsync(nbr_ptr, p->nbr_ptr, sizeof(int) * (p->sum_loc + p->K), cudaMemcpyDeviceToHost, s));
        if (nbr) {
            std::vector<uint16_t> tmp(p->sum_edges);
            DDG_CU(cudaMemcpyAsync(tmp.data(), p->nbr, sizeof(uint16_t) * p->sum_edges, cudaMemcpyDeviceToHost, s));
            DDG_CU(cudaStreamSynchronize(s));
            for (long long e = 0; e < p->sum_edges; ++e) nbr[e] = tmp[e];
        }
        DDG_CU(cudaStreamSynchronize(s));
        return DDG_OK;
    });
}

int32_t ddg_coarse_download(ddg_problem *p, double *A0, double *A0_inv) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && p->K > 0, "no partition");
        DDG_TRY(use_device(p->ctx));
        cudaStream_t s = p->stream;
        size_t bytes = sizeof(double) * p->K * p->K;
        if (A0) DDG_CU(cudaMemcpyAsync(A0, p->A0, bytes, cudaMemcpyDeviceToHost, s));
        if (A0_inv) DDG_CU(cudaMemcpyAsync(A0_inv, p->A0inv, bytes, cudaMemcpyDeviceToHost, s));
        DDG_CU(cudaStreamSynchronize(s));
        return DDG_OK;
    });
}

// ------------------------------------------------------------------ model
int32_t ddg_model_create(ddg_ctx *c, int32_t kbar, int32_t d, float alpha, const float *w, size_t n_w,
                         uint64_t seed, ddg_model **out) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(c && out, "NULL argument");
        REQUIRE(d == 5 || d == DSS_D || d == 20, "latent size d must be 5, 10 or 20");
        REQUIRE(kbar >= 1 && kbar <= 256, "kbar must be in [1, 256]");
        size_t per = (size_t)(11 * d * d + 15 * d + 1);
        REQUIRE(n_w == per * kbar, "n_w must be kbar * (11 d^2 + 15 d + 1)");
        DDG_TRY(use_device(c));
        ddg_model *m = new ddg_model();
        m->ctx = c;
        m->kbar = kbar;
        m->d = d;
        m->alpha = alpha;
        m->n_w = n_w;
        int32_t st = dalloc(c, m->allocs, &m->w, n_w);
        if (st == DDG_OK) {
            if (w) {
                cudaError_t e = cudaMemcpy(m->w, w, sizeof(float) * n_w, cudaMemcpyHostToDevice);
                if (e != cudaSuccess) {
                    set_error(cudaGetErrorString(e));
                    st = DDG_CUDA_ERROR;
                }
            } else {
                st = model_xavier(m, seed);
            }
        }
        if (st == DDG_OK && d == DSS_D) st = model_pack(m);  // layouts of schedules 0-4 (d = 10)
        if (st != DDG_OK) {
            dfree_all(c, m->allocs);
            delete m;
            return st;
        }
        *out = m;
        return DDG_OK;
    });
}

int32_t ddg_model_destroy(ddg_model *m) {
    return api_guard([&]() -> int32_t {
        if (!m) return DDG_OK;
        cudaSetDevice(m->ctx->device);
        cudaStreamSynchronize(m->ctx->stream);
        dfree_all(m->ctx, m->allocs);
        delete m;
        return DDG_OK;
    });
}

int32_t ddg_model_get_weights(ddg_model *m, float *w, size_t n_w) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(m && w && n_w == m->n_w, "bad arguments");
        DDG_TRY(use_device(m->ctx));
        DDG_CU(cudaMemcpy(w, m->w, sizeof(float) * n_w, cudaMemcpyDeviceToHost));
        return DDG_OK;
    });
}

int32_t ddg_model_set_weights(ddg_model *m, const float *w, size_t n_w) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(m && w && n_w == m->n_w, "bad arguments");
        DDG_TRY(use_device(m->ctx));
        DDG_CU(cudaMemcpy(m->w, w, sizeof(float) * n_w, cudaMemcpyHostToDevice));
        if (m->d == DSS_D) {  // schedule 5 reads the flat weights directly
            DDG_TRY(model_host_layouts(m));
            DDG_CU(cudaMemcpy(m->packed, m->packed_host.data(), sizeof(float) * m->packed_host.size(),
                              cudaMemcpyHostToDevice));
        }
        return DDG_OK;
    });
}

// ------------------------------------------------------------------ preconditioner and solver
int32_t ddg_setup_precond(ddg_problem *p, int32_t kind, const ddg_model *model, uint32_t flags) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && p->assembled, "problem not assembled");
        REQUIRE(kind == DDG_NONE || kind == DDG_DDM_LU || kind == DDG_DDM_GNN, "unknown preconditioner kind");
        REQUIRE(kind == DDG_NONE || p->K > 0, "preconditioner needs a partition");
        REQUIRE(kind != DDG_DDM_GNN || model, "DDM-GNN needs a model");
        REQUIRE(!model || model->ctx == p->ctx, "model belongs to another context");
        DDG_TRY(use_device(p->ctx));
        ddg_ctx *c = p->ctx;
        dfree_all(c, p->a_kry);
        p->kr_m = 0;
        dfree_all(c, p->a_pre);
        chunk_free(p);
        p->kind = DDG_NONE;
        p->flags = flags;
        p->model = model;
        if (kind == DDG_NONE) return DDG_OK;
        DDG_TRY(dalloc(c, p->a_pre, &p->s, p->K));
        DDG_TRY(dalloc(c, p->a_pre, &p->y, p->K));
        DDG_TRY(dalloc(c, p->a_pre, &p->wc, p->K));
        DDG_TRY(dalloc(c, p->a_pre, &p->corr, p->sum_k));
        if (kind == DDG_DDM_LU) {
            DDG_TRY(lu_build(p));
        } else {
            DDG_TRY(dss_check_capacity(p));
            DDG_TRY(dss_select_weights(p, (flags & DDG_BF16_WEIGHTS) != 0));
            // latents: d planes of sum_loc (schedules 0-2, 5) or rows of 12 floats, h then c (schedules 3, 4)
            const size_t hl = (size_t)std::max(DSS_HROW, model->d) * p->sum_loc;
            DDG_TRY(dalloc(c, p->a_pre, &p->dss_h, hl));
            DDG_TRY(dalloc(c, p->a_pre, &p->dss_h2, hl));
            DDG_TRY(dalloc(c, p->a_pre, &p->dss_c, p->sum_loc));
            p->kind = kind;
            DDG_TRY(dss_autotune(p));
        }
        p->kind = kind;
        return DDG_OK;
    });
}

int32_t ddg_precondition(ddg_problem *p, const double *r_dev, double *z_dev, ddg_stream stream) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && p->assembled && r_dev && z_dev, "bad arguments");
        DDG_TRY(use_device(p->ctx));
        cudaStream_t s = stream ? (cudaStream_t)stream : p->stream;
        return precond_apply(p, r_dev, z_dev, s, false, nullptr, nullptr);
    });
}

int32_t ddg_local_corrections(ddg_problem *p, const double *r_dev, double *corr_dev, double *s_dev,
                              ddg_stream stream) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && p->kind != DDG_NONE && r_dev && corr_dev && s_dev, "bad arguments");
        DDG_TRY(use_device(p->ctx));
        cudaStream_t s = stream ? (cudaStream_t)stream : p->stream;
        return precond_apply(p, r_dev, nullptr, s, true, corr_dev, s_dev);
    });
}

int32_t ddg_apply_A(ddg_problem *p, const double *x_dev, double *y_dev, ddg_stream stream) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && p->assembled && x_dev && y_dev, "bad arguments");
        DDG_TRY(use_device(p->ctx));
        cudaStream_t s = stream ? (cudaStream_t)stream : p->stream;
        return spmv(p, x_dev, y_dev, s);
    });
}

int32_t ddg_train_local_model(ddg_problem *p, ddg_model *m, const ddg_train_opts *o, ddg_train_report *report) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && p->assembled && p->K > 0 && m && o, "training needs an assembled, partitioned problem and a model");
        REQUIRE(m->ctx == p->ctx, "model belongs to another context");
        REQUIRE(o->steps >= 0 && o->batch >= 1 && o->harvest_iters >= 2 && o->lr > 0.f, "bad training options");
        REQUIRE(p->max_loc <= DSS_MAX_NODES, "local graphs too large for the GNN kernels");
        REQUIRE(m->d == DSS_D, "the training kernels are compiled for d = 10");
        DDG_TRY(use_device(p->ctx));
        int32_t st = train_local_model(p, m, o, report);
        return st;
    });
}

int32_t ddg_train_loss_grad(ddg_problem *p, ddg_model *m, const double *r_dev, const int32_t *graphs, int32_t nb,
                            double *loss, float *grad) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && p->assembled && p->K > 0 && m && r_dev && graphs && nb >= 1 && loss, "bad arguments");
        for (int b = 0; b < nb; ++b) REQUIRE(graphs[b] >= 0 && graphs[b] < p->K, "graph index out of range");
        REQUIRE(m->d == DSS_D, "the training kernels are compiled for d = 10");
        DDG_TRY(use_device(p->ctx));
        return train_loss_grad(p, m, r_dev, graphs, nb, loss, grad);
    });
}

int32_t ddg_fcg_history(ddg_problem *p, double *rel_host, int32_t n, int32_t *count) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && count && n >= 0 && (rel_host || n == 0), "bad arguments");
        DDG_TRY(use_device(p->ctx));
        *count = p->khist_n;
        const int m = std::min(n, p->khist_n);
        if (m > 0) {
            DDG_CU(cudaMemcpyAsync(rel_host, p->khist, sizeof(double) * m, cudaMemcpyDeviceToHost, p->stream));
            DDG_CU(cudaStreamSynchronize(p->stream));
        }
        return DDG_OK;
    });
}

int32_t ddg_fcg_solve(ddg_problem *p, const double *x0, double rtol, int32_t max_iter, int32_t m_trunc,
                      double *x_host, ddg_solve_report *report) {
    return api_guard([&]() -> int32_t {
        API_BEGIN;
        REQUIRE(p && p->assembled, "problem not assembled");
        REQUIRE(rtol > 0.0 && max_iter >= 1, "rtol must be > 0 and max_iter >= 1");
        DDG_TRY(use_device(p->ctx));
        return fcg_solve(p, x0, rtol, max_iter, m_trunc, x_host, report);
    });
}

}  // extern "C"
