// Device-wide primitives used by the setup stage: exclusive scan, merge sort of
// index arrays under a total order, deterministic FP64 sum; plus allocation
// through the context's HBM budget and the per-thread error message.
#include "ddg_internal.cuh"

#include <cstdio>

namespace ddg {

static thread_local std::string g_last_error;
static unsigned long long g_launches = 0;

void note_launches(int n) { __atomic_fetch_add(&g_launches, (unsigned long long)n, __ATOMIC_RELAXED); }
unsigned long long launch_count() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

void set_error(const std::string &msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }
const char *last_error_cstr() { return g_last_error.c_str(); }

int32_t dmalloc(ddg_ctx *ctx, Allocs &a, void **p, size_t bytes) {
    if (ctx->budget && ctx->in_use.load() + bytes > ctx->budget) {
        set_error("HBM budget exceeded: " + std::to_string(ctx->in_use.load() + bytes) + " > " +
                  std::to_string(ctx->budget) + " bytes");
        return DDG_OOM;
    }
    cudaError_t e = a.use_stream ? cudaMallocAsync(p, bytes, a.stream) : cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        return DDG_OOM;
    }
    a.ptrs.push_back(*p);
    a.sizes.push_back(bytes);
    ctx->in_use += bytes;
    return DDG_OK;
}

void dfree_all(ddg_ctx *ctx, Allocs &a) {
    for (size_t i = 0; i < a.ptrs.size(); ++i) {
        if (a.use_stream) cudaFreeAsync(a.ptrs[i], a.stream); else cudaFree(a.ptrs[i]);
        ctx->in_use -= a.sizes[i];
    }
    a.ptrs.clear();
    a.sizes.clear();
}

int32_t check_status(ddg_problem *p, const char *where) {
    int st = 0;
    DDG_CU(cudaMemcpyAsync(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    DDG_CU(cudaStreamSynchronize(p->stream));
    if (st == 0) return DDG_OK;
    DDG_CU(cudaMemsetAsync(p->d_status, 0, sizeof(int), p->stream));
    std::string w(where);
    if (st & ST_BAD_MESH) {
        set_error(w + ": degenerate/inverted triangle or node degree above the cap");
        return DDG_BAD_MESH;
    }
    if (st & ST_TIMEOUT) {
        set_error(w + ": a kernel's bounded wait for its data ran out");
        return DDG_TIMEOUT;
    }
    if (st & ST_TOO_LARGE) {
        set_error(w + ": a list exceeds a kernel's capacity");
        return DDG_TOO_LARGE;
    }
    set_error(w + ": invalid input values");
    return DDG_INVALID_ARG;
}

// ------------------------------------------------------------------ scan
constexpr int SCAN_T = 1024, SCAN_ITEMS = 4, SCAN_TILE = SCAN_T * SCAN_ITEMS;

__global__ void __launch_bounds__(SCAN_T) k_scan_tile(const int *in, int *out, int *sums, int n) {
    __shared__ int sh[32];
    long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int tsum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        tsum += v[k];
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = sh[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    int excl = x - tsum + (warp > 0 ? sh[warp - 1] : 0);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = excl;
        excl += v[k];
    }
    if (threadIdx.x == SCAN_T - 1) sums[blockIdx.x] = excl;
}

__global__ void k_scan_add(int *out, const int *offs, int n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / SCAN_TILE];
}

// exclusive scan of n ints; in == out allowed; total_host (if not NULL) receives the sum
static int32_t scan_rec(const int *in, int *out, int n, int *total_dev, cudaStream_t s) {
    int nb = cdiv(n, SCAN_TILE);
    Scratch sc(s);
    int *sums = nullptr, *offs = nullptr;
    DDG_CU(sc.get(&sums, nb + 1));
    k_scan_tile<<<nb, SCAN_T, 0, s>>>(in, out, sums, n);
    DDG_LAUNCH_CHECK();
    if (nb == 1) {
        DDG_CU(cudaMemcpyAsync(total_dev, sums, sizeof(int), cudaMemcpyDeviceToDevice, s));
    } else {
        DDG_CU(sc.get(&offs, nb));
        DDG_TRY(scan_rec(sums, offs, nb, total_dev, s));
        k_scan_add<<<cdiv(n, 256), 256, 0, s>>>(out, offs, n);
        DDG_LAUNCH_CHECK();
    }
    return DDG_OK;
}

int32_t scan_exclusive(ddg_ctx *ctx, const int *in, int *out, int n, int *total_host, cudaStream_t s) {
    (void)ctx;
    Scratch sc(s);
    int *tot = nullptr;
    DDG_CU(sc.get(&tot, 1));
    if (n == 0) {
        DDG_CU(cudaMemsetAsync(tot, 0, sizeof(int), s));
    } else {
        DDG_TRY(scan_rec(in, out, n, tot, s));
    }
    if (total_host) {
        DDG_CU(cudaMemcpyAsync(total_host, tot, sizeof(int), cudaMemcpyDeviceToHost, s));
        DDG_CU(cudaStreamSynchronize(s));
    }
    return DDG_OK;
}

// ------------------------------------------------------------------ merge sort
// Bottom-up merge of sorted runs.  Keys are distinct under the order, so an
// element's new position is its rank inside its run plus its rank in the partner run.
template <class Cmp>
__global__ void k_merge_pass(const int *in, int *out, int n, int width, Cmp cmp) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int e = in[i];
    long long start = ((long long)i / (2LL * width)) * 2LL * width;
    int mid = (int)min((long long)n, start + width);
    int end = (int)min((long long)n, start + 2LL * width);
    int lo, hi, base;
    if (i < mid) {
        lo = mid; hi = end; base = i - (int)start;
    } else {
        lo = (int)start; hi = mid; base = i - mid;
    }
    int first = lo;
    while (lo < hi) {
        int m = (lo + hi) >> 1;
        if (cmp.less(in[m], e)) lo = m + 1; else hi = m;
    }
    out[start + base + (lo - first)] = e;
}

__global__ void k_iota(int *a, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = i;
}

template <class Cmp>
static int32_t merge_sort(int *idx, int n, Cmp cmp, cudaStream_t s) {
    if (n <= 1) return DDG_OK;
    Scratch sc(s);
    int *tmp = nullptr;
    DDG_CU(sc.get(&tmp, n));
    int *a = idx, *b = tmp;
    for (long long w = 1; w < n; w *= 2) {
        k_merge_pass<<<cdiv(n, 256), 256, 0, s>>>(a, b, n, (int)w, cmp);
        DDG_LAUNCH_CHECK();
        int *t = a; a = b; b = t;
    }
    if (a != idx) DDG_CU(cudaMemcpyAsync(idx, a, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    return DDG_OK;
}

struct PointCmp {
    const double *xy;
    int axis;
    __device__ bool less(int a, int b) const {
        double a0 = xy[2 * a + axis], b0 = xy[2 * b + axis];
        if (a0 != b0) return a0 < b0;
        double a1 = xy[2 * a + 1 - axis], b1 = xy[2 * b + 1 - axis];
        if (a1 != b1) return a1 < b1;
        return a < b;
    }
};

struct PairCmp {
    const int *major, *minor;
    __device__ bool less(int a, int b) const {
        if (major[a] != major[b]) return major[a] < major[b];
        if (minor[a] != minor[b]) return minor[a] < minor[b];
        return a < b;
    }
};

// out_idx = ids 0..n-1 ordered by (coord[axis], coord[1-axis], id)
int32_t sort_points(ddg_ctx *ctx, const double *xy, int n, int axis, int *out_idx, cudaStream_t s) {
    (void)ctx;
    if (n == 0) return DDG_OK;
    k_iota<<<cdiv(n, 256), 256, 0, s>>>(out_idx, n);
    DDG_LAUNCH_CHECK();
    return merge_sort(out_idx, n, PointCmp{xy, axis}, s);
}

// out_idx = ids 0..n-1 ordered by (major, minor, id)
int32_t sort_pairs(ddg_ctx *ctx, const int *major, const int *minor, int n, int *out_idx, cudaStream_t s) {
    (void)ctx;
    if (n == 0) return DDG_OK;
    k_iota<<<cdiv(n, 256), 256, 0, s>>>(out_idx, n);
    DDG_LAUNCH_CHECK();
    return merge_sort(out_idx, n, PairCmp{major, minor}, s);
}

// ------------------------------------------------------------------ sum
constexpr int RED_BLOCKS = 296, RED_T = 256;

__global__ void __launch_bounds__(RED_T) k_sum_partial(const double *in, int n, double *part) {
    __shared__ double sh[32];
    double v = 0.0;
    for (long long i = (long long)blockIdx.x * RED_T + threadIdx.x; i < n; i += (long long)RED_BLOCKS * RED_T) v += in[i];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__global__ void __launch_bounds__(RED_T) k_sum_final(const double *part, int np, double *out) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < np; i += RED_T) v += part[i];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) *out = v;
}

int32_t reduce_sum(ddg_ctx *ctx, const double *in, int n, double *out_dev, cudaStream_t s) {
    (void)ctx;
    Scratch sc(s);
    double *part = nullptr;
    DDG_CU(sc.get(&part, RED_BLOCKS));
    k_sum_partial<<<RED_BLOCKS, RED_T, 0, s>>>(in, n, part);
    DDG_LAUNCH_CHECK();
    k_sum_final<<<1, RED_T, 0, s>>>(part, RED_BLOCKS, out_dev);
    DDG_LAUNCH_CHECK();
    return DDG_OK;
}

}  // namespace ddg
