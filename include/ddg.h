/*
 * ddg.h - C ABI of the DDM-GNN solver library (libddg.so).
 *
 * The library solves the P1 finite-element Poisson-Dirichlet problem
 * -Lap(u) = f in Omega, u = g on the boundary (Section II, Eqs. 1-2) with
 * flexible conjugate gradients preconditioned by the paper's two-level
 * additive Schwarz method, whose local solves are either exact (DDM-LU,
 * Eq. 7) or one inference of a Deep Statistical Solver GNN (DDM-GNN,
 * Section III-A, Eqs. 13-16; architecture Section III-B, Eqs. 18-22).
 * Everything after the upload runs in the library's CUDA kernels on one GPU.
 *
 * Conventions
 *  - Every call returns an int32_t status (DDG_OK = 0 or a negative code).
 *    No call aborts, throws or traps; after a failure ddg_last_error()
 *    returns a message for the calling thread.  Besides the codes listed
 *    with each call, any call may return DDG_OOM when host memory runs out
 *    and DDG_INTERNAL for another host-side failure.
 *  - Handles are opaque and owned by the caller, who frees them with the
 *    matching *_destroy call.  A problem or model must be destroyed before
 *    its context.
 *  - Host arrays passed in are copied before the call returns; the caller
 *    keeps ownership.  Host arrays passed out are written, never kept.
 *  - Device pointers (ddg_precondition, ddg_apply_A, ddg_local_corrections)
 *    are borrowed: they must live on the context's device and are used in
 *    stream order on the stream given.  NULL selects the context's own
 *    stream, which is non-blocking: it does not synchronise with the legacy
 *    default stream, so pass cudaStreamLegacy to run on that one.
 *  - Indices are int32, zero-based.  "free" nodes are the mesh nodes that are
 *    not Dirichlet nodes, numbered in ascending mesh order.
 *  - A context and everything created from it is not thread-safe, except
 *    ddg_submit, ddg_poll and ddg_serve_stats, which any thread may call.
 */
#ifndef DDG_H
#define DDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ddg_ctx ddg_ctx;
typedef struct ddg_problem ddg_problem;
typedef struct ddg_model ddg_model;
typedef void *ddg_stream; /* a cudaStream_t */

enum ddg_status {
    DDG_OK = 0,
    DDG_INVALID_ARG = -1,   /* bad size, NULL pointer, call out of order */
    DDG_OOM = -2,           /* device allocation failed or HBM budget exceeded */
    DDG_CUDA_ERROR = -3,    /* a CUDA runtime call failed */
    DDG_NOT_CONVERGED = -4, /* max_iter reached */
    DDG_BREAKDOWN = -5,     /* p.q <= 0 or a non-finite scalar in the Krylov loop */
    DDG_BUSY = -6,          /* ddg_submit: the admission queue is full */
    DDG_TIMEOUT = -7,       /* a kernel's bounded wait (about one second) ran out; the context stays usable */
    DDG_PENDING = -8,       /* ddg_poll: the request has not finished yet */
    DDG_BAD_MESH = -9,      /* degenerate or inverted triangle, or a node of too high degree */
    DDG_TOO_LARGE = -10,    /* a subdomain or node list beyond a kernel's on-chip capacity */
    DDG_INTERNAL = -11      /* a host-side failure other than memory (a thread that cannot be started) */
};

enum ddg_precond_kind { DDG_NONE = 0, DDG_DDM_LU = 1, DDG_DDM_GNN = 2 };

enum ddg_precond_flags {
    DDG_COARSE = 1u,      /* add the Nicolaides coarse correction (two-level, Eq. 7) */
    DDG_POU_PROLONG = 2u, /* glue local corrections with partition-of-unity weights instead of R_i^T */
    DDG_BF16_WEIGHTS = 4u /* DDM-GNN: run with the model's weights rounded to bfloat16 (nearest, ties to even);
                             latents and arithmetic stay FP32.  Not in the paper: a storage-precision variant */
};

typedef struct ddg_solve_report {
    int32_t status;            /* DDG_OK, DDG_NOT_CONVERGED or DDG_BREAKDOWN */
    int32_t iterations;        /* FCG iterations taken */
    double rel_residual;       /* recursive |r| / |b| at exit */
    double true_rel_residual;  /* |b - A x| / |b| recomputed at exit (FP64) */
    double solve_ms;           /* device time of the Krylov loop (CUDA events on the solve stream) */
    double precond_ms;         /* device time of all preconditioner applications */
    double local_ms;           /* device time of the local-solve kernel alone (GNN or band solves) */
    int32_t local_launches;    /* kernel launches of the local solves inside the loop */
    int32_t launches;          /* all kernel launches of the library inside the loop */
    int32_t local_applies;     /* local-solve applications (one per iteration) */
    int32_t gnn_schedule;      /* 0: one launch per application, 1: one launch per message-passing block,
                                  2: as 1 with the graphs cut into chunks of at most 2 * gnn_chunk_t nodes,
                                  3: equal-work ranges of the concatenated graphs, packed FP32 (the default
                                  pick), 4: as 3 with the per-node products on the tensor cores through
                                  tensor memory, 5: any latent size d in {5, 10, 20}, 6: as 4 with
                                  warp-synchronous tensor-core MMAs; -1 for DDM-LU */
    int32_t gnn_chunk_t;       /* threads per CTA of the chunked schedules 2-6 (0 otherwise) */
} ddg_solve_report;

/* ---- context --------------------------------------------------------- */

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the
 * device memory the context's objects may hold (0 = no cap).  Errors:
 * DDG_INVALID_ARG (no such device), DDG_CUDA_ERROR. */
int32_t ddg_create(int32_t device, size_t hbm_budget_bytes, ddg_ctx **out);
int32_t ddg_destroy(ddg_ctx *ctx);
/* Message of the calling thread's last failure (empty string if none). */
const char *ddg_last_error(void);
/* Device memory currently held by the context's objects, in bytes. */
int32_t ddg_memory_in_use(ddg_ctx *ctx, size_t *bytes);
/* The context's own CUDA stream (a cudaStream_t), on which every call
 * without an explicit stream runs; lets a caller record events around calls. */
int32_t ddg_get_stream(ddg_ctx *ctx, ddg_stream *out);
/* Number of kernel launches the library has issued in this process so far. */
int32_t ddg_launch_count(uint64_t *out);

/* ---- mesh and assembly (Section II, Eqs. 1-2) ------------------------ */

/* Upload a triangle mesh: xy[2*n_nodes] FP64 coordinates (x0, y0, x1, ...),
 * tri[3*n_tri] vertex ids, counter-clockwise.  dirichlet[n_nodes] marks the
 * Dirichlet nodes (nonzero = Dirichlet); NULL selects the endpoints of the
 * boundary edges (edges in exactly one triangle).  The device builds the node
 * adjacency, checks every triangle's orientation and the mean edge length
 * h_bar.  Errors: DDG_INVALID_ARG, DDG_BAD_MESH (area <= 0, a node in more
 * than 32 triangles or with more than 32 neighbours), DDG_OOM. */
int32_t ddg_mesh_upload(ddg_ctx *ctx, int32_t n_nodes, const double *xy, int32_t n_tri,
                        const int32_t *tri, const uint8_t *dirichlet, ddg_problem **out);
int32_t ddg_problem_destroy(ddg_problem *p);

/* Assemble A_ff and b_f - A_fD g_D for the paper's data family (Section IV-A,
 * Eqs. 24-25): f = r1 (x-1)^2 + r2 y^2 + r3 and g = r4 x^2 + r5 y^2 + r6 xy +
 * r7 x + r8 y + r9, r = r[0..8].  The load is integrated exactly through f's
 * P2 interpolant.  Any earlier partition or preconditioner is dropped. */
int32_t ddg_assemble_poly(ddg_problem *p, const double r[9]);
/* The same with nodal f[n_nodes] (consistent P1 mass matrix) and nodal
 * g[n_nodes] (used at the Dirichlet nodes). */
int32_t ddg_assemble_nodal(ddg_problem *p, const double *f, const double *g);

/* Sizes: info[0] n_nodes, [1] n_tri, [2] n_free, [3] nnz of A_ff, [4] K,
 * [5] sum of subdomain sizes, [6] sum of local graph sizes (with halo),
 * [7] sum of local graph edges, [8] largest local graph, [9] h_bar as the
 * bit pattern of an FP64 value.  Unknown entries are -1. */
int32_t ddg_problem_info(ddg_problem *p, int64_t info[10]);

/* Download the assembled free-free CSR (rowptr[n_free+1], col[nnz], val[nnz])
 * and the right-hand side b[n_free].  Any output pointer may be NULL. */
int32_t ddg_matrix_download(ddg_problem *p, int32_t *rowptr, int32_t *col, double *val, double *b);

/* ---- decomposition (Section II-A; Section IV-A) ------------------------ */

/* Split the free nodes into K parts by recursive coordinate bisection (or
 * take part_or_NULL[n_free], values in [0, K)), grow each part by
 * overlap_layers adjacency layers of the A_ff graph, and build the
 * partition-of-unity weights 1/multiplicity, the local DSS graphs and the
 * coarse matrix A_0 = Z^T A Z.  Errors: DDG_INVALID_ARG, DDG_TOO_LARGE (a
 * node in more than 32 subdomains), DDG_OOM. */
int32_t ddg_partition(ddg_problem *p, int32_t K, int32_t overlap_layers, const int32_t *part_or_null);

/* Download part[n_free], sub_ptr[K+1], sub_idx[sum k_i] (ascending free ids
 * of every subdomain) and mult[n_free].  NULL outputs are skipped. */
int32_t ddg_partition_download(ddg_problem *p, int32_t *part, int32_t *sub_ptr, int32_t *sub_idx, int32_t *mult);

/* Download the local graphs: loc_ptr[K+1] offsets of every graph's nodes,
 * n_int[K], loc_node[sum n_loc] mesh ids (unknowns ascending, then halo
 * ascending), nbr_ptr[sum n_loc + K] per-graph CSR offsets (graph i's slice
 * starts at loc_ptr[i] + i), nbr[sum edges] local neighbour ids: every mesh
 * neighbour for an unknown, the unknown neighbours for a halo node.
 * NULL outputs are skipped. */
int32_t ddg_graph_download(ddg_problem *p, int32_t *loc_ptr, int32_t *n_int, int32_t *loc_node,
                           int32_t *nbr_ptr, int32_t *nbr);

/* Download A_0 (K*K, row-major) and its inverse as the setup computed it. */
int32_t ddg_coarse_download(ddg_problem *p, double *A0, double *A0_inv);

/* ---- DSS model (Section III-B; Table 2) -------------------------------- */

/* Create a model with kbar blocks of latent size d and ResNet step alpha.
 * d = 10 (the paper's setting) runs on every GNN schedule, the training
 * kernels and BF16 weights; d = 5 and d = 20 (the other columns of Table 2's
 * sweep) run inference on the generic schedule 5.  w (n_w = kbar * (11 d^2 +
 * 15 d + 1) floats, layout per block row-major W[out][in]: Phi_out W1[d][2d+3]
 * b1[d] W2[d][d] b2[d]; Phi_in the same; Psi W1[d][3d+1] b1[d] W2[d][d] b2[d];
 * D W1[d][d] b1[d] W2[1][d] b2[1]) or NULL for Xavier-uniform matrices and
 * zero biases drawn from SplitMix64(seed).  Errors: DDG_INVALID_ARG (n_w
 * mismatch, d not in {5, 10, 20}). */
int32_t ddg_model_create(ddg_ctx *ctx, int32_t kbar, int32_t d, float alpha, const float *w, size_t n_w,
                         uint64_t seed, ddg_model **out);
int32_t ddg_model_destroy(ddg_model *m);
int32_t ddg_model_get_weights(ddg_model *m, float *w, size_t n_w);

/* Replace the model's weights by w[n_w] (host, copied; flat layout of
 * ddg_model_create).  Problems set up with this model see the new weights at
 * their next GNN launch; the Adam moments of ddg_train_local_model are kept.
 * Errors: DDG_INVALID_ARG (n_w differs from the model's). */
int32_t ddg_model_set_weights(ddg_model *m, const float *w, size_t n_w);

/* Training of the DSS local solver (Section III-B, Eq. 23; optimiser of
 * Section IV-B) on the local problems of problem p's own decomposition
 * (Section IV-A): p is set up with DDG_DDM_LU (it stays so), preconditioned
 * CG runs for harvest_iters - 1 iterations, and every stored residual r^n
 * gives K samples c = R_i r^n / |R_i r^n| on the local graphs.  Each step
 * draws `batch` samples, evaluates sum_k mean((R_i A R_i^T r_hat^k - c)^2)
 * with hand-written forward and backward kernels, clips the gradient to
 * global norm `clip`, and takes an Adam step (beta 0.9/0.999, eps 1e-8);
 * the learning rate drops x0.1 after 8 windows of 50 steps without a 0.1 %
 * improvement.  The model's weights are updated in place; its Adam moments
 * persist in the model, so successive calls on different problems continue
 * one optimisation.  Errors:
 * DDG_INVALID_ARG (no partition, bad options, a model with d != 10), DDG_OOM,
 * DDG_CUDA_ERROR. */
typedef struct ddg_train_opts {
    int32_t steps;          /* optimiser steps */
    int32_t batch;          /* samples per step */
    float lr;               /* Adam learning rate (1e-2 in Section IV-B) */
    float clip;             /* gradient-norm clip (1e-2 in Section IV-B; <= 0 disables) */
    int32_t harvest_iters;  /* residuals kept per problem: r_0 .. r_{harvest_iters - 1} */
    uint64_t seed;          /* SplitMix64 seed of the sample draws */
} ddg_train_opts;

typedef struct ddg_train_report {
    int32_t samples;        /* local problems available (K x stored residuals) */
    int32_t steps;
    double loss_first;      /* batch loss of the first and of the last step */
    double loss_last;
    double ms;              /* device time of harvest and training */
    double lr_final;
} ddg_train_report;

int32_t ddg_train_local_model(ddg_problem *p, ddg_model *m, const ddg_train_opts *opts, ddg_train_report *report);

/* The training loss and its gradient for the given local graphs, each with
 * c = R_i r / |R_i r| from one device residual r_dev (n_free FP64): loss =
 * mean over graphs[0..nb) of sum_k mean((R_i A R_i^T r_hat^k - c)^2), grad =
 * its gradient w.r.t. the flat weights (n_w floats, layout of
 * ddg_model_create).  For checking the hand-written backward (d = 10 models). */
int32_t ddg_train_loss_grad(ddg_problem *p, ddg_model *m, const double *r_dev, const int32_t *graphs, int32_t nb,
                            double *loss, float *grad);

/* ---- preconditioner and solver --------------------------------------- */

/* Build the preconditioner of the given kind on the current partition:
 * DDG_DDM_LU factorises every R_i A R_i^T (banded FP64 Cholesky);
 * DDG_DDM_GNN uses `model` (kept by reference; it must outlive its use).
 * flags: DDG_COARSE, DDG_POU_PROLONG, DDG_BF16_WEIGHTS.  The GNN schedule
 * is tuned here (timed on the right-hand side, cached per decomposition
 * shape class); local graphs of more than 2,048 nodes run on the chunked
 * schedules; a model with d != 10 runs on schedule 5.  Errors:
 * DDG_INVALID_ARG (no partition, missing model, DDG_BF16_WEIGHTS with
 * d != 10), DDG_TOO_LARGE (a local graph beyond 65,535 nodes), DDG_OOM. */
int32_t ddg_setup_precond(ddg_problem *p, int32_t kind, const ddg_model *model, uint32_t flags);

/* z = M^-1 r for device vectors r_dev, z_dev of n_free FP64 (Eqs. 13-16 for
 * DDM-GNN, Eq. 7 for DDM-LU, z = r for DDG_NONE). */
int32_t ddg_precondition(ddg_problem *p, const double *r_dev, double *z_dev, ddg_stream stream);

/* The local corrections alone: s_dev[K] = |R_i r| and corr_dev[sum k_i] (in
 * sub_idx order) = |R_i r| r~_i for DDM-GNN or (R_i A R_i^T)^-1 R_i r for DDM-LU. */
int32_t ddg_local_corrections(ddg_problem *p, const double *r_dev, double *corr_dev, double *s_dev,
                              ddg_stream stream);

/* y = A_ff x for device vectors of n_free FP64. */
int32_t ddg_apply_A(ddg_problem *p, const double *x_dev, double *y_dev, ddg_stream stream);

/* y = A_ff x and *xy_dev = x . y (FP64, deterministic) without allocating any
 * device memory, for callers that cannot call cudaMalloc (inside a stream
 * capture owned by someone else, under an allocator that forbids allocations
 * after start-up, or in a loop that cannot afford an allocation).  No passage
 * of the paper corresponds to this call; it exists for those callers.
 * x_dev, y_dev: n_free FP64 device vectors; xy_dev: one FP64 on the device.
 * Scratch is a 512 KiB array compiled into the library, which every GPU that
 * loads the library holds until the process exits; n_free may be at most
 * 16,777,216 (DDG_TOO_LARGE beyond).  The first call on a device looks up the
 * array's device address, so make that first call before any stream capture;
 * the address is kept for the life of the process, so do not use this call
 * after a device reset in the same process.
 * All calls share the array: calls that overlap on the GPU race and their dot
 * products are then wrong; order them on one stream.  Errors:
 * DDG_INVALID_ARG, DDG_TOO_LARGE, DDG_CUDA_ERROR. */
int32_t ddg_apply_A_dot_noalloc(ddg_problem *p, const double *x_dev, double *y_dev, double *xy_dev,
                                ddg_stream stream);

/* Solve A_ff x = b_f by flexible CG (truncation m_trunc >= 1; m_trunc = 1
 * reproduces PCG for a fixed SPD preconditioner) from x0 (host, n_free, or
 * NULL = 0) until |r| / |b| < rtol or max_iter iterations.  x_host[n_nodes]
 * receives the full nodal solution (g on Dirichlet nodes).  Before the first
 * iteration: b = 0 returns x = 0 (whatever x0) and a start vector with
 * |b - A x0| / |b| < rtol returns x0, both with zero iterations and DDG_OK.
 * Returns the report's status: DDG_OK, DDG_NOT_CONVERGED, DDG_BREAKDOWN, or DDG_TIMEOUT
 * when a kernel gave up a bounded wait during the solve (the context stays
 * usable). */
int32_t ddg_fcg_solve(ddg_problem *p, const double *x0, double rtol, int32_t max_iter, int32_t m_trunc,
                      double *x_host, ddg_solve_report *report);

/* The residual history of the problem's last ddg_fcg_solve: rel_host[i] =
 * |r_(i+1)| / |b| (the recursive residual after iteration i + 1), for the
 * first min(n, *count) iterations; *count = iterations recorded (the first
 * 1,048,576 at most).  Host buffer, caller-owned.  Errors: DDG_INVALID_ARG. */
int32_t ddg_fcg_history(ddg_problem *p, double *rel_host, int32_t n, int32_t *count);

/* ---- serving (continuous batching of independent solves) ------------- */

typedef struct ddg_solve_opts {
    int32_t kind;            /* DDG_DDM_GNN, DDG_DDM_LU or DDG_NONE */
    uint32_t flags;          /* DDG_COARSE, DDG_POU_PROLONG, DDG_BF16_WEIGHTS */
    const ddg_model *model;  /* for DDG_DDM_GNN; must outlive the request */
    int32_t K;               /* subdomains; 0 = round(n_free / 1000) */
    int32_t overlap;         /* overlap layers */
    double rtol;
    int32_t max_iter;
    int32_t m_trunc;
} ddg_solve_opts;

typedef struct ddg_serve_summary {
    uint64_t completed, failed, pending, active;
    uint64_t reserved_bytes;  /* device memory estimated for the admitted requests */
    uint64_t device_bytes;    /* device memory held by the context */
    double p50_ms, p99_ms;    /* latency from submit to result, over completed requests */
    double solves_per_s;      /* completed requests / (last completion - first submit) */
} ddg_serve_summary;

/* Queue the solve of -Lap(u) = f, u = g (data family of Eqs. 24-25, r[0..8])
 * on the given mesh (copied) and return a ticket.  A scheduler thread owned by
 * the context admits queued requests in arrival order while fewer than
 * max_active run and their estimated device memory fits the context's HBM
 * budget, sets each up on a stream of its own and advances all running
 * solves a batch of iterations at a time, so their GPU work overlaps (or, with
 * fused GNN launches, one iteration per step; see ddg_serve_config).
 * Thread-safe with ddg_poll and ddg_serve_stats.  Errors: DDG_INVALID_ARG,
 * DDG_BUSY (the admission queue holds max_pending requests). */
int32_t ddg_submit(ddg_ctx *ctx, int32_t n_nodes, const double *xy, int32_t n_tri, const int32_t *tri,
                   const double r[9], const ddg_solve_opts *opts, uint64_t *ticket);
/* DDG_PENDING while the request is queued or running; afterwards its final
 * status (DDG_OK, DDG_NOT_CONVERGED, DDG_BREAKDOWN or a set-up error), the
 * report (solve_ms = wall time from admission to the result) and, if x_host
 * is not NULL, the nodal solution (n_nodes).  A ticket is collected once. */
int32_t ddg_poll(ddg_ctx *ctx, uint64_t ticket, ddg_solve_report *report, double *x_host);
/* Most requests in flight at once (default 64), most requests waiting for
 * admission (default 65536; ddg_submit returns DDG_BUSY beyond it), and whether
 * concurrent DDM-GNN requests share fused GNN launches (fuse_gnn = 1: each step
 * advances every member of a group by one FCG iteration, the members'
 * subdomains in one launch per message-passing block; 0, the default: every
 * request runs its own kernels on its own stream, its FCG periods replayed as
 * CUDA graphs, and the GPU overlaps the requests).  Results are the same
 * either way.  The settings apply to requests submitted or started after the
 * call. */
int32_t ddg_serve_config(ddg_ctx *ctx, int32_t max_active, int32_t fuse_gnn, int32_t max_pending);
int32_t ddg_serve_stats(ddg_ctx *ctx, ddg_serve_summary *out);

#ifdef __cplusplus
}
#endif

#endif /* DDG_H */
