// Internal declarations of libddg: object layouts, error plumbing, device helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <atomic>
#include <exception>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/ddg.h"

namespace ddg {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
void clear_error();

#define DDG_CU(call)                                                                      \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            ddg::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));          \
            return DDG_CUDA_ERROR;                                                        \
        }                                                                                 \
    } while (0)

#define DDG_TRY(call)                   \
    do {                                \
        int32_t s_ = (call);            \
        if (s_ != DDG_OK) return s_;    \
    } while (0)

// Runs the body of an entry point so that no C++ exception crosses the C ABI: a failed host
// allocation returns DDG_OOM, any other exception (a thread that cannot be started, say)
// DDG_INTERNAL, each with its message.
template <class F>
int32_t api_guard(F &&body) noexcept {
    try {
        return body();
    } catch (const std::bad_alloc &) {
        set_error("host memory allocation failed");
        return DDG_OOM;
    } catch (const std::length_error &e) {
        set_error(std::string("host allocation too large: ") + e.what());
        return DDG_OOM;
    } catch (const std::exception &e) {
        set_error(std::string("internal error: ") + e.what());
        return DDG_INTERNAL;
    } catch (...) {
        set_error("internal error");
        return DDG_INTERNAL;
    }
}

// every launch site is followed by DDG_LAUNCH_CHECK (or DDG_LAUNCHES(n) for n launches)
void note_launches(int n);
unsigned long long launch_count();
#define DDG_LAUNCHES(n)           \
    do {                          \
        ddg::note_launches(n);    \
        DDG_CU(cudaGetLastError()); \
    } while (0)
#define DDG_LAUNCH_CHECK() DDG_LAUNCHES(1)

// device status bits raised by bounded checks inside kernels
enum : int {
    ST_BAD_MESH = 1,      // non-positive triangle area, node degree over the cap
    ST_TOO_LARGE = 2,     // list longer than a kernel's local capacity
    ST_BAD_INPUT = 4,     // user partition value out of range
    ST_TIMEOUT = 8,       // a bounded wait ran out
};

constexpr int MAX_NODE_TRI = 32;   // triangles around one node
constexpr int MAX_NODE_NBR = 32;   // mesh neighbours of one node
constexpr int MAX_MEMBERSHIP = 32; // subdomains holding one node
constexpr int DSS_D = 10;          // latent size compiled into the GNN kernel
constexpr int DSS_THREADS = 512;
constexpr int DSS_HROW = 12;        // floats per latent row of the fused schedule (h[10], c, pad)
constexpr int DSS_MAX_NODES = 2048; // local graph nodes (unknowns + halo) per CTA

struct Server;  // request scheduler (serve.cu)

// ---------------------------------------------------------------- allocation
// device allocations of one stage; stream-ordered (no device-wide synchronisation on
// free) when `stream` is set, as for the buffers of a problem
struct Allocs {
    std::vector<void *> ptrs;
    std::vector<size_t> sizes;
    cudaStream_t stream = nullptr;
    bool use_stream = false;
};

}  // namespace ddg

struct ddg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0;
    bool pdl = true;  // programmatic dependent launches between GNN blocks (DDG_NO_PDL=1 turns them off)
    std::atomic<size_t> in_use{0};
    ddg::Server *server = nullptr;  // started by the first ddg_submit
    std::mutex server_mu;
    std::mutex tune_mu;             // guards `tuned` (set-up may run on the scheduler thread)
    // GNN schedule chosen by the autotuner, cached per decomposition shape class: K in quarter
    // octaves, mean graph size in steps of 64 nodes, largest graph in steps of 128 nodes
    struct Tuned {
        long long K, nodes, max_loc;  // the three classes
        int sched, T;
    };
    std::vector<Tuned> tuned;
};

struct ddg_model {
    ddg_ctx *ctx = nullptr;
    int kbar = 0, d = 0;
    float alpha = 0.f;
    size_t n_w = 0;
    float *w = nullptr;       // flat weights as given (device)
    float *packed = nullptr;  // per-block padded layout read by the GNN kernel (device)
    size_t packed_per_block = 0;
    std::vector<float> packed_host;  // the same packed weights on the host (kernel-parameter copies)
    std::vector<float> fused_host;   // composed per-block layout of the fused GNN kernel (kernel parameters)
    float *tc_w = nullptr;           // per-block tensor-core weight images of schedule 4 (device)
    float *mma_w = nullptr;          // per-block warp-MMA weight fragments of schedule 6 (device)
    float *adam_m = nullptr, *adam_v = nullptr;  // Adam moments, kept across training calls
    long long adam_t = 0;
    ddg::Allocs allocs;
};

// chunked GNN schedule: graphs cut into chunks of at most 2 * T nodes (see dss.cu)
struct ChunkPlan {
    int T = 0, nchunks = 0, max_need = 0;
    size_t max_smem = 0;  // schedule 3: largest per-CTA shared memory of the plan
    bool global = false;  // schedules 3, 4: chunks are ranges of the concatenated graphs' nodes, sized to fill
                          // the GPU evenly; own nodes sorted by message count, neighbour kind in bit 15
    bool tc = false;      // schedule 4: at most T own and TC_NEED needed nodes per chunk (tensor-core kernel)
    int *gid = nullptr;   // global: graph of every local node (sum_loc)
    int4 *info = nullptr; // global: per own slot {node, corr index or -1, free index of r or -1,
                          //   graph | out-messages << 24}
    int *c_graph = nullptr, *c_n0 = nullptr, *c_own = nullptr, *c_need_off = nullptr, *c_need_n = nullptr;
    int *need = nullptr, *c_adj_off = nullptr, *adj_ptr = nullptr, *c_adj_base = nullptr;
    uint16_t *adj = nullptr;
    uint2 *adjx = nullptr;  // schedule 4: per adjacency entry {chunk-local neighbour, edge length |d| as float
                            //   bits}, each own node's unknown neighbours first
    ddg::Allocs allocs;
};

struct ddg_problem {
    ddg_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;  // the context's stream, or a stream of its own (served requests)
    bool own_stream = false;
    int *d_status = nullptr;  // device status word (bits ST_*)

    // mesh (stage "mesh")
    int n = 0, t = 0;
    double *xy = nullptr;      // [2n]
    int *tri = nullptr;        // [3t]
    uint8_t *dir = nullptr;    // [n] Dirichlet flags
    int *ntri_ptr = nullptr, *ntri_idx = nullptr;  // node -> incident triangles (ascending)
    int *adj_ptr = nullptr, *adj_idx = nullptr;    // node -> mesh neighbours (ascending)
    int n_edges = 0;
    double hbar = 0.0;
    int nf = 0;
    int *free_id = nullptr;    // [n], -1 on Dirichlet nodes
    int *free_node = nullptr;  // [nf]
    double *xy_free = nullptr; // [2 nf]
    ddg::Allocs a_mesh;

    // matrix (stage "matrix")
    bool assembled = false;
    int nnz = 0;
    int *rowptr = nullptr, *col = nullptr;
    double *val = nullptr, *b = nullptr;
    // the same matrix in sliced ELLPACK for the SpMV (krylov.cu): slices of 32 rows, rows sorted
    // by decreasing length within windows of 256; slot k holds row sl_perm[k]; entry e of the
    // slot's row at sl_ptr[k / 32] + 32 e + k % 32 (padding: column = the row, value 0)
    int n_slices = 0;
    int *sl_perm = nullptr, *sl_len = nullptr, *sl_ptr = nullptr, *sl_col = nullptr;
    double *sl_val = nullptr;
    double *g = nullptr;       // [n] Dirichlet values (0 on free nodes)
    double bnorm = 0.0;
    ddg::Allocs a_matrix;

    // partition (stage "part")
    int K = 0, delta = 0;
    int *part = nullptr;                     // [nf]
    int *mem_ptr = nullptr, *mem_idx = nullptr; // node -> subdomains (ascending)
    int *mult = nullptr;                     // [nf]
    double *inv_mult = nullptr;              // [nf] 1 / mult
    int *sub_ptr = nullptr, *sub_idx = nullptr; // subdomain -> free ids (ascending)
    int *inv_pos = nullptr;                  // mem slot -> position in sub_idx
    long long sum_k = 0;
    // local graphs
    int *loc_ptr = nullptr, *loc_nint = nullptr, *loc_node = nullptr;
    float2 *loc_xy = nullptr;                // (x - centre) / h_bar, FP32
    int *nbr_ptr = nullptr;                  // per graph: n_loc + 1 offsets (graph i starts at loc_ptr[i] + i)
    int *nbr_off = nullptr;                  // [K] start of graph i's neighbour slice
    uint16_t *nbr = nullptr;
    long long sum_loc = 0, sum_edges = 0;
    int max_loc = 0, max_edges = 0;
    int *lpt_order = nullptr;                // subdomains by decreasing graph size
    double *A0 = nullptr, *A0inv = nullptr;  // [K*K]
    ddg::Allocs a_part;

    // preconditioner (stage "precond")
    int kind = DDG_NONE;
    uint32_t flags = 0;
    const ddg_model *model = nullptr;
    int *lu_perm = nullptr;     // [sum_k] band position -> position in sub_idx slice
    int *lu_pos = nullptr;      // [sum_k] position in sub_idx slice -> band position
    int *lu_bw = nullptr;       // [K]
    long long *lu_off = nullptr; // [K+1] start of each band factor
    double *lu_band = nullptr;
    double *lu_bandT = nullptr;      // the factor's transpose, same storage (backward solves)
    long long *lu_toff = nullptr;    // [K+1] start of each subdomain's diagonal-tile inverses
    double *lu_tinv = nullptr;       // 32 x 32 inverse of every diagonal tile of L, row-major
    int lu_kmax = 0;
    double *s = nullptr, *y = nullptr, *wc = nullptr, *corr = nullptr;
    // GNN weights in use: the model's, or (DDG_BF16_WEIGHTS) this problem's copies rounded to bfloat16
    bool w_bf16 = false;
    float *bf16_packed_dev = nullptr;
    float *bf16_tc_dev = nullptr;   // schedule-4 weight images of the rounded weights
    float *bf16_mma_dev = nullptr;  // schedule-6 weight fragments of the rounded weights
    std::vector<float> bf16_packed_host, bf16_fused_host;
    bool dss_whole_graph = true;  // every local graph fits one CTA (schedules 0 and 1 allowed)
    int dss_sched = 0;          // GNN schedule: 0 one persistent launch, 1 one launch per block, 2 chunked per block,
                                // 3 chunked per block with composed weights and packed two-lane FP32,
                                // 4 as 3 with the per-node matrix products on the tensor cores,
                                // 5 any latent size d in {5, 10, 20} (flat weights, schedule 2's chunks)
    float *dss_h = nullptr, *dss_c = nullptr;  // latents and c between launches (schedules 1, 2)
    float *dss_h2 = nullptr;    // second latent buffer (schedule 2)
    ChunkPlan chunk;
    ddg::Allocs a_pre;

    // Krylov workspace (stage "krylov")
    int *hflag_pinned = nullptr;  // host copy of the Krylov flags (pinned)
    int kr_m = 0;
    double *kx = nullptr, *kr = nullptr, *kz = nullptr, *kP = nullptr, *kQ = nullptr, *kscal = nullptr;
    double *kpart = nullptr;   // block partials of reductions
    int *kflag = nullptr;
    double *khist = nullptr;   // |r| / |b| after every iteration of the last solve
    int khist_cap = 0, khist_n = 0;
    ddg::Allocs a_hist;
    ddg::Allocs a_kry;
};

namespace ddg {

// allocation through the context's budget
int32_t dmalloc(ddg_ctx *ctx, Allocs &a, void **p, size_t bytes);
template <class T>
int32_t dalloc(ddg_ctx *ctx, Allocs &a, T **p, size_t n) {
    return dmalloc(ctx, a, reinterpret_cast<void **>(p), (n ? n : 1) * sizeof(T));
}
void dfree_all(ddg_ctx *ctx, Allocs &a);

// Stream-ordered temporaries of one host scope.  Every pointer taken with get() is freed on
// the stream when the scope ends, on every return path (the early returns of DDG_TRY and
// DDG_CU included); drop() frees one earlier.  A pointer taken here is never passed to
// cudaFreeAsync directly.
class Scratch {
  public:
    explicit Scratch(cudaStream_t s) : s_(s) {}
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    ~Scratch() {
        for (void *q : ptrs_) cudaFreeAsync(q, s_);
    }
    template <class T>
    cudaError_t get(T **p, size_t n) {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(p), sizeof(T) * n, s_);
        if (e == cudaSuccess) ptrs_.push_back(*p);
        return e;
    }
    cudaError_t drop(void *q) {
        for (size_t i = 0; i < ptrs_.size(); ++i)
            if (ptrs_[i] == q) {
                ptrs_.erase(ptrs_.begin() + (long)i);
                return cudaFreeAsync(q, s_);
            }
        return cudaSuccess;
    }

  private:
    cudaStream_t s_;
    std::vector<void *> ptrs_;
};

int32_t check_status(ddg_problem *p, const char *where);
const char *last_error_cstr();
int32_t problem_create(ddg_ctx *c, int n_nodes, const double *xy, int n_tri, const int *tri, const uint8_t *dirichlet,
                       cudaStream_t stream, bool own_stream, ddg_problem **out);
void server_stop(ddg_ctx *c);

// primitives (prims.cu)
int32_t scan_exclusive(ddg_ctx *ctx, const int *in, int *out, int n, int *total_host, cudaStream_t s);
int32_t sort_points(ddg_ctx *ctx, const double *xy, int n, int axis, int *out_idx, cudaStream_t s);
int32_t sort_pairs(ddg_ctx *ctx, const int *major, const int *minor, int n, int *out_idx, cudaStream_t s);
int32_t reduce_sum(ddg_ctx *ctx, const double *in, int n, double *out_dev, cudaStream_t s);

// stages
int32_t mesh_build(ddg_problem *p, const uint8_t *dirichlet_host);
int32_t assemble(ddg_problem *p, const double *r9, const double *f_nodal, const double *g_nodal);
int32_t partition_build(ddg_problem *p, int K, int delta, const int *part_host);
int32_t coarse_build(ddg_problem *p);
int32_t lu_build(ddg_problem *p);
int32_t precond_apply(ddg_problem *p, const double *r, double *z, cudaStream_t s, bool corrections_only,
                      double *corr_out, double *s_out);
int32_t spmv(ddg_problem *p, const double *x, double *y, cudaStream_t s);
int32_t sell_build(ddg_problem *p);  // the sliced ELLPACK copy of A_ff (after assembly)
int32_t model_pack(ddg_model *m);
int32_t model_host_layouts(ddg_model *m);
int32_t dss_select_weights(ddg_problem *p, bool bf16);  // rebuilds packed_host and fused_host from the device flat weights
int32_t dss_launch_args(ddg_problem *p, const double *r, const int *stop, cudaStream_t s);
int32_t dss_check_capacity(ddg_problem *p);
int32_t dss_autotune(ddg_problem *p);
int32_t chunk_build(ddg_problem *p, int T);
struct ChunkArgs;
int32_t chunk_build_global(ddg_problem *p, int T, bool tc);
// schedule 4 (dss_tc.cu): per-node matrix products of the GNN on the tensor cores
constexpr int TC_T = 128;            // threads of a CTA, and own nodes of a chunk at most
constexpr int TC_NEED = 256;         // needed nodes of a chunk at most (two 128-row tiles)
constexpr int TCW_FLOATS = 3328;     // floats of one block's tensor-core weight images (three GEMMs)
constexpr size_t TC_SMEM = 47104;    // dynamic shared memory of a schedule-4 CTA (at most four per SM)
constexpr int TC_CTAS_PER_SM = 4;    // schedule-4 CTAs an SM holds (4 x 128 tensor-memory columns)
void tc_weight_image(const float *fused, int kbar, std::vector<float> &img);
int32_t tc_ctas_per_sm(int *out);
int32_t dss_tc_launch(ddg_problem *p, const ChunkArgs &a, const float *fused_host, const float *tc_w, cudaStream_t s);
// schedule 6 (dss_mma.cu): schedule 4's chunks, per-node products as warp-synchronous tensor-core MMAs
constexpr int MMA_W_FLOATS = 3072;  // floats of one block's MMA weight fragments (four products)
void mma_weight_image(const float *fused, int kbar, std::vector<float> &img);
int32_t dss_mma_launch(ddg_problem *p, const ChunkArgs &a, const float *fused_host, const float *mma_w,
                       cudaStream_t s);
// schedule 5 (dss_d.cu): latent sizes d = 5, 10, 20 from the flat weights, on schedule 2's chunks
constexpr int DSS_D_CHUNK_T = 128;
int32_t dss_d_launch(ddg_problem *p, const ChunkArgs &a, cudaStream_t s);
// fused GNN steps over several problems (request loop): schedule 3 with chunk width GROUP_T
constexpr int GROUP_T = 128;
int32_t dss_group_prepare(ddg_problem *p);
bool dss_group_compatible(const ddg_problem *a, const ddg_problem *b);
size_t dss_group_args_bytes();
int32_t dss_group_launch(ddg_problem *const *ps, const double *const *rs, const int *const *stops, int n,
                         ChunkArgs *dev_args, bool upload, cudaStream_t s);
void chunk_free(ddg_problem *p);
int32_t model_xavier(ddg_model *m, uint64_t seed);
int32_t lu_apply_launch(ddg_problem *p, const double *r, const int *stop, cudaStream_t s);
int32_t fcg_solve(ddg_problem *p, const double *x0, double rtol, int max_iter, int m, double *x_host,
                  ddg_solve_report *rep, double *record = nullptr);
int32_t fcg_solve_record(ddg_problem *p, int iters, double *record, int *stored);
struct FcgRun;
FcgRun *fcg_new();
void fcg_delete(FcgRun *r);
int32_t fcg_begin(FcgRun *r, ddg_problem *p, const double *x0, double rtol, int max_iter, int m);
int32_t fcg_launch_batch(FcgRun *r);
int32_t fcg_check(FcgRun *r, bool blocking, bool *ready, bool *done);
int32_t fcg_end(FcgRun *r, double *x_host, ddg_solve_report *rep);
// fused-step mode: group_pre (restriction, coarse solve) and group_post (gluing and the FCG
// kernels, then the iteration counter advances) bracket a fused GNN launch over several runs;
// group_mark queues the flag copy that fcg_check observes
int32_t fcg_group_pre(FcgRun *r);
int32_t fcg_group_post(FcgRun *r);
int32_t fcg_group_mark(FcgRun *r);
int fcg_group_since_mark(const FcgRun *r);
int fcg_iterations_launched(const FcgRun *r);
int fcg_max_iter(const FcgRun *r);
const double *fcg_residual(const FcgRun *r);
const int *fcg_flag(const FcgRun *r);
int32_t train_local_model(ddg_problem *p, ddg_model *m, const ddg_train_opts *o, ddg_train_report *rep);
int32_t train_loss_grad(ddg_problem *p, ddg_model *m, const double *r_dev, const int *graphs_host, int nb,
                        double *loss, float *grad_host);

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// device helpers ---------------------------------------------------------
__device__ __forceinline__ void raise_status(int *st, int bit) { atomicOr(st, bit); }

template <class T>
__device__ __forceinline__ void insertion_sort(T *a, int n) {
    for (int i = 1; i < n; ++i) {
        T v = a[i];
        int j = i - 1;
        while (j >= 0 && a[j] > v) {
            a[j + 1] = a[j];
            --j;
        }
        a[j + 1] = v;
    }
}

// deterministic block sum of one double per thread (blockDim.x multiple of 32, <= 1024)
__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (warp == 0) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;  // valid in thread 0
}

}  // namespace ddg
