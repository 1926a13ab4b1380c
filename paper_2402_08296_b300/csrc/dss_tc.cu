// Schedule 4 of the batched Deep Statistical Solver inference (Section III-B, Eqs. 18-22):
// chunks of the concatenated local graphs as in schedule 3 (one launch per message-passing
// block), with every per-node matrix product on the fifth-generation tensor cores and only the
// edge messages on the CUDA cores.
//
// A CTA of 128 threads loops over chunks of at most 128 own nodes (one thread per own node) and
// 256 needed nodes (own nodes first, then their neighbours outside the chunk).  Per chunk:
//   GEMM1 (every needed node): [h, x, y, c, d_out, d_in, 1] (16 inputs) -> 64 outputs: the
//     neighbour projections Wb h + We_xy x of both edge MLPs (Eqs. 18-19, interleaved in the
//     order the edge loop reads them from shared memory), and for own nodes the negated
//     first-layer terms -(Wa h + b1 - We_xy x_j) of both messages and the h, c and degree part
//     of Psi's hidden layer (Eq. 20, the message MLPs' second layers composed into it);
//   edge loop (CUDA cores): with q = pb + We_|d| |d| and relu(pa + q) = max(q, -pa) + pa,
//     S = sum over the neighbours of max(q, -pa), plus (messages) * pa afterwards; each
//     node's neighbour list holds the unknowns first, so out-messages (to unknowns only) and
//     in-messages (from all neighbours) run as two plain loops, and the edge length |d| comes
//     precomputed with the neighbour's index;
//   GEMM2: [S_out, S_in] (24 inputs) accumulated onto the hidden-layer columns of GEMM1;
//   GEMM3: [relu(hidden), 1] (16 inputs) -> alpha (Psi_W2 relu + Psi_b2), the residual update;
//   the decoder (Eq. 22) of the last block on the CUDA cores.
// Each GEMM is one tcgen05.mma chain (kind::tf32) per 128-row tile, issued by one thread from
// shared-memory operands into FP32 accumulators in tensor memory and read back with tcgen05.ld,
// whose 32x32b shape hands every thread the row of the node it owns.  FP32 accuracy from the
// TF32 tensor cores by a three-term split: the tensor core truncates its FP32 inputs to TF32,
// so x W = x W_hi + x_lo W_hi + x W_lo up to terms below 2^-20 relative, with W_hi = W
// truncated to TF32 and W_lo = W - W_hi (both exact in FP32) and x_lo = x - trunc(x), each
// product one more K-concatenated term of the same accumulator.
//
// Operands are K-major without swizzling: 8-row x 16-byte core matrices, the K-chunks of a
// row group contiguous (leading-dimension byte offset 128 between core matrices along K,
// stride-dimension byte offset K/4 * 128 between row groups).  The block's three weight images
// come with one bulk copy per CTA and launch.  Tensor memory: 128 columns per CTA for the
// whole launch (GEMM1 tile 0 at column 0 with N = 64, GEMM2 onto its columns 48-63; tile 1,
// outside neighbours only, at column 64 with N = 32; GEMM3 at column 96 with N = 16).  The
// CTA's shared memory keeps at most four CTAs on an SM, so the 512 columns of an SM always
// suffice and an allocation never waits.  Every wait on a barrier is bounded (about one
// second), after which the CTA raises ST_TIMEOUT, waits once more for the operations in
// flight, frees its tensor memory and returns.
#include "dss_layout.cuh"

#include <cstring>

namespace ddg {

// ---------------------------------------------------------------- weight image of one block
constexpr int TC_KA = 16, TC_NA = 64;   // GEMM1: K, N
constexpr int TC_K2 = 24, TC_N2 = 16;   // GEMM2
constexpr int TC_K3 = 16, TC_N3 = 16;   // GEMM3
constexpr int TCW_B1 = 0;                               // hi [64][16], then lo
constexpr int TCW_B2 = TCW_B1 + 2 * TC_NA * TC_KA;      // 2048: hi [16][24], then lo
constexpr int TCW_B3 = TCW_B2 + 2 * TC_N2 * TC_K2;      // 2816: hi [16][16], then lo
static_assert(TCW_B3 + 2 * TC_N3 * TC_K3 == TCW_FLOATS, "weight image size");
static_assert((TCW_FLOATS * 4) % 16 == 0, "the image is one bulk copy of whole 16-byte pieces");
// output columns of GEMM1 (tile 0)
constexpr int C_PB = 0, C_NPA = 20, C_HID = 48;

// shared memory of a CTA (bytes).  Region R (32 KB) holds in turn: GEMM1's operand rows X and
// XL (256 rows each); the needed nodes' projections (256 x 80 bytes); GEMM2's operand rows
// (128 x 24 floats, and the low parts); GEMM3's (128 x 16).  Then the weight images, barriers
// and the tensor-memory address.
constexpr int TC_OFF_XL = TC_NEED * TC_KA * 4;        // 16384
constexpr int TC_OFF_A2L = TC_T * TC_K2 * 4;          // 12288
constexpr int TC_OFF_A3L = TC_T * TC_K3 * 4;          // 8192
constexpr int TC_OFF_W = 2 * TC_OFF_XL;               // 32768
constexpr int TC_OFF_BAR = TC_OFF_W + TCW_FLOATS * 4; // 46080: MMA barrier, weight barrier, TMEM address
static_assert(TC_NEED * 80 <= TC_OFF_W && 2 * TC_OFF_A2L <= TC_OFF_W, "the overlays fit region R");
static_assert(TC_OFF_BAR + 24 <= (int)TC_SMEM, "shared memory layout");
static_assert(5 * (TC_SMEM + 1024) > 228 * 1024, "at most four schedule-4 CTAs per SM (4 x 128 TMEM columns)");

constexpr uint32_t TMEM_COLS = 128;

// float offset of element (r, k) of a K-major matrix with K columns, in core-matrix order
__host__ __device__ __forceinline__ int tc_core(int r, int k, int K) {
    return ((r >> 3) * (K >> 2) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

static float tf32_high(float w) {
    uint32_t b;
    std::memcpy(&b, &w, 4);
    b &= 0xffffe000u;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

// element (r, k) of the B operand at `off` (N rows of K), high part then low part
static void put_w(float *img, int off, int N, int K, int r, int k, float w) {
    const float hi = tf32_high(w);
    img[off + tc_core(r, k, K)] = hi;
    img[off + N * K + tc_core(r, k, K)] = w - hi;
}

// The B operands of every block from the composed per-block layout of schedule 3
// (dss_layout.cuh), row = output, column = input.
//  B1 columns: 0-9 h, 10 x, 11 y, 12 c, 13 d_out, 14 d_in, 15 one.  Rows 0-19 the neighbour
//     projections, out/in pairs interleaved as in shared memory; 20-29 -pa_out; 30-39 -pa_in;
//     48-57 the GEMM's part of Psi's hidden layer; the rest zero.
//  B2 columns: 0-9 S_out, 10-19 S_in; rows 0-9 the hidden layer (Psi_W1 W2_out | Psi_W1 W2_in).
//  B3 columns: 0-9 relu(hidden), 10 one; rows 0-9 alpha Psi_W2 | alpha Psi_b2.
void tc_weight_image(const float *fused, int kbar, std::vector<float> &img) {
    img.assign((size_t)kbar * TCW_FLOATS, 0.f);
    for (int b = 0; b < kbar; ++b) {
        const float *f = fused + (size_t)b * F_FLOATS;
        float *o = img.data() + (size_t)b * TCW_FLOATS;
        auto w1 = [&](int r, int k, float w) { put_w(o, TCW_B1, TC_NA, TC_KA, r, k, w); };
        for (int r = 0; r < 2 * D; ++r) {
            for (int i = 0; i < D; ++i) w1(C_PB + r, i, f[F_HB + i * 2 * D + r]);
            w1(C_PB + r, 10, f[F_XB + r]);
            w1(C_PB + r, 11, f[F_XB + 2 * D + r]);
        }
        for (int q = 0; q < D; ++q) {
            const int ro = C_NPA + q, ri = C_NPA + D + q, rh = C_HID + q;
            for (int i = 0; i < D; ++i) {
                w1(ro, i, -f[F_HA + i * 3 * D + q]);
                w1(ri, i, -f[F_HA + i * 3 * D + D + q]);
                w1(rh, i, f[F_HA + i * 3 * D + 2 * D + q]);
            }
            w1(ro, 10, -f[F_NXA + q]);
            w1(ro, 11, -f[F_NXA + 2 * D + q]);
            w1(ro, 15, -f[F_BA + q]);
            w1(ri, 10, -f[F_NXA + D + q]);
            w1(ri, 11, -f[F_NXA + 3 * D + q]);
            w1(ri, 15, -f[F_BA + D + q]);
            w1(rh, 12, f[F_VC + q]);
            w1(rh, 13, f[F_VO + q]);
            w1(rh, 14, f[F_VI + q]);
            w1(rh, 15, f[F_BA + 2 * D + q]);
            for (int i = 0; i < D; ++i) {
                put_w(o, TCW_B2, TC_N2, TC_K2, q, i, f[F_MO + i * D + q]);
                put_w(o, TCW_B2, TC_N2, TC_K2, q, D + i, f[F_MI + i * D + q]);
                put_w(o, TCW_B3, TC_N3, TC_K3, q, i, f[F_P2 + i * D + q]);
            }
            put_w(o, TCW_B3, TC_N3, TC_K3, q, 10, f[F_PB2 + q]);
        }
    }
}

// ---------------------------------------------------------------- tcgen05 helpers
// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M = 128
__host__ __device__ constexpr uint32_t tc_idesc(int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
}

// shared-memory matrix descriptor: K-major, no swizzling, core matrices as described above
__device__ __forceinline__ uint64_t tc_desc(const void *base, int K) {
    const uint32_t a = smem_u32(base);
    return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
           ((uint64_t)(((uint32_t)(K / 4) * 128u) >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// D (+)= A B^T over `steps` K-steps of 8 with the three-term split (one 32-byte K-step advances
// a descriptor's address field by 2 core matrices = 256 bytes = 16 units); acc0 = 0 starts D
// from zero, 1 accumulates onto what D holds
__device__ __forceinline__ void tc_gemm3(uint32_t d, uint64_t ax, uint64_t axl, uint64_t bh, uint64_t bl, int steps,
                                         uint32_t idesc, int acc0) {
    int acc = acc0;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const uint64_t a = t == 1 ? axl : ax, b = t == 2 ? bl : bh;
        for (int s = 0; s < steps; ++s) {
            tc_mma(d, a + 16ull * s, b + 16ull * s, idesc, acc);
            acc = 1;
        }
    }
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tf32_low(float x) { return x - __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

// row r of an A operand (K inputs) and of its low part
template <int K>
__device__ __forceinline__ void tc_put_row(float *X, float *XL, int r, const float (&v)[K]) {
#pragma unroll
    for (int c = 0; c < K / 4; ++c) {
        const int o = tc_core(r, 4 * c, K);
        *reinterpret_cast<float4 *>(X + o) = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
        *reinterpret_cast<float4 *>(XL + o) = make_float4(tf32_low(v[4 * c]), tf32_low(v[4 * c + 1]),
                                                          tf32_low(v[4 * c + 2]), tf32_low(v[4 * c + 3]));
    }
}

// max of each lane with the matching lane of b; a NaN in either stays NaN (max.NaN)
__device__ __forceinline__ f2_t f2_max(f2_t a, f2_t b) {
    float a0, a1, b0, b1;
    f2_unpack(a, a0, a1);
    f2_unpack(b, b0, b1);
    float r0, r1;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r0) : "f"(a0), "f"(b0));
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r1) : "f"(a1), "f"(b1));
    return f2_pack(r0, r1);
}

// whether the phase of the given parity of an mbarrier has completed (no waiting)
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// 16-byte shared-memory load at a 32-bit shared address
__device__ __forceinline__ float4 lds4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}

// what staging a chunk's GEMM1 rows reads from global memory, per thread: its two rows'
// latent vectors and coordinates, and its own node's record and adjacency range
struct ChunkRows {
    int own, nn;
    float4 h[2][3];
    float c[2];
    float2 xy[2];
    int4 inf;
    int e0, e1;
};

__device__ __forceinline__ void chunk_rows_load(const ChunkArgs &a, int q, int tid, bool first, ChunkRows &r) {
    r.own = a.c_own[q];
    r.nn = a.c_need_n[q];
    const int *need = a.need + a.c_need_off[q];
    const float4 *rows = reinterpret_cast<const float4 *>(a.h_in);
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const int u = tid + rr * TC_T;
        r.h[rr][0] = r.h[rr][1] = r.h[rr][2] = make_float4(0.f, 0.f, 0.f, 0.f);
        r.xy[rr] = make_float2(0.f, 0.f);
        if (u < r.nn) {
            const int node = need[u];
            r.xy[rr] = a.loc_xy[node];
            if (!first) {
                r.h[rr][0] = rows[3 * (size_t)node];
                r.h[rr][1] = rows[3 * (size_t)node + 1];
                r.h[rr][2] = rows[3 * (size_t)node + 2];
            }
        }
        r.c[rr] = r.h[rr][2].z;
    }
    r.inf = make_int4(0, -1, 0, 0);
    r.e0 = r.e1 = 0;
    if (tid < r.own) {
        r.inf = a.info[a.c_n0[q] + tid];
        const int *aptr = a.adj_ptr + a.c_adj_off[q];
        r.e0 = aptr[tid];
        r.e1 = aptr[tid + 1];
    }
}

// ---------------------------------------------------------------- the kernel
// Shared-memory phases of one chunk, with the barrier between them: (stage X) | GEMM1 | (Pb)
// | edge loop | (A2) | GEMM2 | (A3) | GEMM3 | epilogue.  The k-th commit of the CTA completes
// phase k & 1 of the MMA barrier.
__global__ void __launch_bounds__(TC_T, 4)
    k_dss_tc(const __grid_constant__ FusedWeights W, const __grid_constant__ ChunkArgs a, const float *wimg,
             int nchunks) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    if (a.stop && *a.stop) return;
    float *X = reinterpret_cast<float *>(tsm);
    float *XL = reinterpret_cast<float *>(tsm + TC_OFF_XL);
    float4 *Pb = reinterpret_cast<float4 *>(tsm);  // over the operand rows once GEMM1 is done
    float *A2 = reinterpret_cast<float *>(tsm);
    float *A2L = reinterpret_cast<float *>(tsm + TC_OFF_A2L);
    float *A3 = reinterpret_cast<float *>(tsm);
    float *A3L = reinterpret_cast<float *>(tsm + TC_OFF_A3L);
    float *Ws = reinterpret_cast<float *>(tsm + TC_OFF_W);
    uint64_t *bar = reinterpret_cast<uint64_t *>(tsm + TC_OFF_BAR);
    uint64_t *wbar = bar + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tsm + TC_OFF_BAR + 16);
    const int tid = threadIdx.x, warp = tid >> 5;
    const f2_t *Wp = reinterpret_cast<const f2_t *>(W.w);
    const bool first = a.first != 0, last = a.last != 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(wbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // the block's weights are set-up data: fetched before waiting for the previous block
        bulk_load(Ws, wimg, TCW_FLOATS * 4, wbar);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
    asm volatile("griddepcontrol.wait;" ::: "memory");

    // the edge-length weights of both messages, kept in registers for every chunk
    f2_t wdo[D / 2], wdi[D / 2];
#pragma unroll
    for (int m = 0; m < D / 2; ++m) {
        wdo[m] = Wp[(F_WEO + 2 * D) / 2 + m];
        wdi[m] = Wp[(F_WEI + 2 * D) / 2 + m];
    }
    uint32_t commits = 0;
    bool ok = true;
    bool weights_waited = false, weights_ok = false;  // thread 0: the weight copy was waited for / landed
    // the CTA's next commit: thread 0 waits (bounded) while the others wait at the barrier, then
    // every thread checks the completed phase once; false (in every thread) if the wait ran out,
    // the weight copy's included
    auto mma_wait = [&]() -> bool {
        const uint32_t par = commits & 1u;
        ++commits;
        bool mine = true;
        if (tid == 0) mine = weights_ok && mbar_wait(bar, par);
        const bool bad = __syncthreads_or(!mine) != 0;
        // every thread sees the completed phase itself (at once: thread 0 saw it before the barrier)
        if (!bad && !mbar_test(bar, par) && !mbar_wait(bar, par)) raise_status(a.status, ST_TIMEOUT);
        tc_fence_after();
        return !bad;
    };

    // the rows of the chunk to be staged next, loaded one chunk ahead: the loads of chunk q's
    // rows are issued while chunk q - gridDim.x waits for its GEMM2 and GEMM3
    ChunkRows pre;
    if (blockIdx.x < nchunks) chunk_rows_load(a, blockIdx.x, tid, first, pre);
    for (int q = blockIdx.x; q < nchunks && ok; q += gridDim.x) {
        const int own = pre.own;
        const int nn = pre.nn;
        const uint2 *ADJ = a.adjx + a.c_adj_base[q];

        // ---- GEMM1 operand rows: row tid (tile 0) and row 128 + tid (tile 1, outside neighbours)
        float h[D], c = 0.f;
        const int4 inf = pre.inf;
        const bool inner = tid < own && inf.y >= 0;
        const int e0 = pre.e0, e1 = pre.e1;
#pragma unroll
        for (int o = 0; o < D; ++o) h[o] = 0.f;
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int u = tid + rr * TC_T;
            if (u >= nn) continue;
            float v[TC_KA], cv = pre.c[rr];
            v[0] = pre.h[rr][0].x; v[1] = pre.h[rr][0].y; v[2] = pre.h[rr][0].z; v[3] = pre.h[rr][0].w;
            v[4] = pre.h[rr][1].x; v[5] = pre.h[rr][1].y; v[6] = pre.h[rr][1].z; v[7] = pre.h[rr][1].w;
            v[8] = pre.h[rr][2].x; v[9] = pre.h[rr][2].y;
            v[10] = pre.xy[rr].x;
            v[11] = pre.xy[rr].y;
            v[12] = v[13] = v[14] = v[15] = 0.f;
            if (u < own) {  // rr == 0: the own node of this thread
                if (first) {
                    const double s = a.s[inf.w & 0xffffff];
                    cv = (inner && s != 0.0) ? (float)(a.r[inf.z] / s) : 0.f;
                }
                v[12] = cv;
                v[13] = (float)((unsigned)inf.w >> 24);
                v[14] = inner ? (float)(e1 - e0) : 0.f;
                v[15] = 1.f;
#pragma unroll
                for (int o = 0; o < D; ++o) h[o] = v[o];
                c = cv;
            }
            tc_put_row<TC_KA>(X, XL, u, v);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            if (!weights_waited) {
                weights_ok = mbar_wait(wbar, 0);
                weights_waited = true;
            }
            if (weights_ok) {
                tc_fence_after();
                const uint64_t bh = tc_desc(Ws + TCW_B1, TC_KA), bl = tc_desc(Ws + TCW_B1 + TC_NA * TC_KA, TC_KA);
                tc_gemm3(tmem, tc_desc(X, TC_KA), tc_desc(XL, TC_KA), bh, bl, TC_KA / 8, tc_idesc(TC_NA), 0);
                if (nn > TC_T)
                    tc_gemm3(tmem + 64u, tc_desc(X + TC_T * TC_KA, TC_KA), tc_desc(XL + TC_T * TC_KA, TC_KA), bh, bl,
                             TC_KA / 8, tc_idesc(32), 0);
            }
            tc_commit(bar);  // arrives when the MMAs above (if any) are done
        }
        if (!(ok = mma_wait())) break;
        // ---- read back: projections of the needed rows into shared memory (over the operand
        // rows, which the completed GEMM no longer reads); the own node's -pa into registers
        f2_t npo[D / 2], npi[D / 2];
        {
            float pv[16], pw[4], v0[16];
            tmem_ld16(tmem + lane + C_PB, pv);
            tmem_ld4(tmem + lane + C_PB + 16, pw);
            tmem_ld16(tmem + lane + C_NPA, v0);  // columns 20-35: -pa_out[10], -pa_in[0..5]
            float v1[4];
            tmem_ld4(tmem + lane + C_NPA + 16, v1);  // columns 36-39: -pa_in[6..9]
            tmem_wait();
            if (tid < nn) {
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    Pb[(size_t)tid * 5 + m] = make_float4(pv[4 * m], pv[4 * m + 1], pv[4 * m + 2], pv[4 * m + 3]);
                Pb[(size_t)tid * 5 + 4] = make_float4(pw[0], pw[1], pw[2], pw[3]);
            }
#pragma unroll
            for (int m = 0; m < D / 2; ++m) npo[m] = f2_pack(v0[2 * m], v0[2 * m + 1]);
            npi[0] = f2_pack(v0[10], v0[11]);
            npi[1] = f2_pack(v0[12], v0[13]);
            npi[2] = f2_pack(v0[14], v0[15]);
            npi[3] = f2_pack(v1[0], v1[1]);
            npi[4] = f2_pack(v1[2], v1[3]);
        }
        if (nn > TC_T) {
            float pv[16], pw[4];
            tmem_ld16(tmem + lane + 64u, pv);
            tmem_ld4(tmem + lane + 80u, pw);
            tmem_wait();
            const int u = TC_T + tid;
            if (u < nn) {
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    Pb[(size_t)u * 5 + m] = make_float4(pv[4 * m], pv[4 * m + 1], pv[4 * m + 2], pv[4 * m + 3]);
                Pb[(size_t)u * 5 + 4] = make_float4(pw[0], pw[1], pw[2], pw[3]);
            }
        }
        __syncthreads();
        // ---- edge messages of the own node: S = sum max(pb + w |d|, -pa), unknown neighbours first
        f2_t so[D / 2], si[D / 2];
#pragma unroll
        for (int m = 0; m < D / 2; ++m) so[m] = si[m] = 0ull;
        const int n_out = min((int)((unsigned)inf.w >> 24), e1 - e0);
        if (tid < own) {
            const uint32_t pb0 = smem_u32(Pb);
            const uint2 *ap = ADJ + e0, *const ae = ADJ + e1, *const au = ADJ + e0 + n_out;
            uint2 nxt = ap < ae ? *ap : make_uint2(0u, 0u);
            for (; ap < au; ++ap) {  // neighbours that are unknowns: out- and in-messages
                const uint2 ent = nxt;
                if (ap + 1 < ae) nxt = ap[1];
                const float dn = __uint_as_float(ent.y);
                const f2_t dn2 = f2_pack(dn, dn);
                const uint32_t pa = pb0 + ent.x * 80u;
                f2_t po[D / 2], pi[D / 2];
#pragma unroll
                for (int m = 0; m < D / 2; ++m) {
                    const float4 t = lds4(pa + 16u * m);
                    po[m] = f2_pack(t.x, t.y);
                    pi[m] = f2_pack(t.z, t.w);
                }
#pragma unroll
                for (int m = 0; m < D / 2; ++m) so[m] = f2_add(so[m], f2_max(f2_fma(wdo[m], dn2, po[m]), npo[m]));
                if (inner) {
#pragma unroll
                    for (int m = 0; m < D / 2; ++m)
                        si[m] = f2_add(si[m], f2_max(f2_fma(wdi[m], dn2, pi[m]), npi[m]));
                }
            }
            if (inner) {
                for (; ap < ae; ++ap) {  // halo neighbours: in-messages only
                    const uint2 ent = nxt;
                    if (ap + 1 < ae) nxt = ap[1];
                    const float dn = __uint_as_float(ent.y);
                    const f2_t dn2 = f2_pack(dn, dn);
                    const uint32_t pa = pb0 + ent.x * 80u;
#pragma unroll
                    for (int m = 0; m < D / 2; ++m) {
                        const float4 t = lds4(pa + 16u * m);
                        si[m] = f2_add(si[m], f2_max(f2_fma(wdi[m], dn2, f2_pack(t.z, t.w)), npi[m]));
                    }
                }
            }
            // relu(pa + q) = max(q, -pa) + pa: add (messages) * pa
            const float fo = -(float)n_out, fi = inner ? -(float)(e1 - e0) : 0.f;
            const f2_t fo2 = f2_pack(fo, fo), fi2 = f2_pack(fi, fi);
#pragma unroll
            for (int m = 0; m < D / 2; ++m) {
                so[m] = f2_fma(fo2, npo[m], so[m]);
                si[m] = f2_fma(fi2, npi[m], si[m]);
            }
        }
        __syncthreads();  // every thread is done with the projections: A2 may overwrite them
        // ---- GEMM2: hidden += (Psi_W1 W2_out) S_out + (Psi_W1 W2_in) S_in
        {
            float v[TC_K2];
#pragma unroll
            for (int m = 0; m < D / 2; ++m) {
                f2_unpack(so[m], v[2 * m], v[2 * m + 1]);
                f2_unpack(si[m], v[D + 2 * m], v[D + 2 * m + 1]);
            }
#pragma unroll
            for (int o = 2 * D; o < TC_K2; ++o) v[o] = 0.f;
            tc_put_row<TC_K2>(A2, A2L, tid, v);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            tc_gemm3(tmem + C_HID, tc_desc(A2, TC_K2), tc_desc(A2L, TC_K2), tc_desc(Ws + TCW_B2, TC_K2),
                     tc_desc(Ws + TCW_B2 + TC_N2 * TC_K2, TC_K2), TC_K2 / 8, tc_idesc(TC_N2), 1);
            tc_commit(bar);
        }
        if (q + (int)gridDim.x < nchunks) chunk_rows_load(a, q + gridDim.x, tid, first, pre);
        if (!(ok = mma_wait())) break;
        // ---- GEMM3: alpha (Psi_W2 relu(hidden) + Psi_b2)
        {
            float hv[16];
            tmem_ld16(tmem + lane + C_HID, hv);
            tmem_wait();
            float v[TC_K3];
#pragma unroll
            for (int o = 0; o < D; ++o) v[o] = relu(hv[o]);
            v[D] = 1.f;
#pragma unroll
            for (int o = D + 1; o < TC_K3; ++o) v[o] = 0.f;
            tc_put_row<TC_K3>(A3, A3L, tid, v);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            tc_gemm3(tmem + 96u, tc_desc(A3, TC_K3), tc_desc(A3L, TC_K3), tc_desc(Ws + TCW_B3, TC_K3),
                     tc_desc(Ws + TCW_B3 + TC_N3 * TC_K3, TC_K3), TC_K3 / 8, tc_idesc(TC_N3), 0);
            tc_commit(bar);
        }
        if (!(ok = mma_wait())) break;
        float dh[16];
        tmem_ld16(tmem + lane + 96u, dh);
        tmem_wait();
        if (tid < own) {
            float hn[D];
#pragma unroll
            for (int o = 0; o < D; ++o) hn[o] = h[o] + dh[o];
            if (last) {
                if (inner) {
                    f2_t dd[D / 2];
#pragma unroll
                    for (int m = 0; m < D / 2; ++m) dd[m] = Wp[F_DB1 / 2 + m];
                    f2_mv<F_DW1, D>(dd, Wp, hn);
                    float y = W.w[F_DB2];
#pragma unroll
                    for (int m = 0; m < D / 2; ++m) {
                        float d0, d1;
                        f2_unpack(dd[m], d0, d1);
                        y = fmaf(W.w[F_DW2 + 2 * m], relu(d0), y);
                        y = fmaf(W.w[F_DW2 + 2 * m + 1], relu(d1), y);
                    }
                    const double s = a.s[inf.w & 0xffffff];
                    a.corr[inf.y] = s == 0.0 ? 0.0 : s * (double)y;
                }
            } else {
                float4 *hrow_out = reinterpret_cast<float4 *>(a.h_out) + 3 * (size_t)inf.x;
                hrow_out[0] = make_float4(hn[0], hn[1], hn[2], hn[3]);
                hrow_out[1] = make_float4(hn[4], hn[5], hn[6], hn[7]);
                hrow_out[2] = make_float4(hn[8], hn[9], c, 0.f);
            }
        }
        tc_fence_before();
        __syncthreads();  // tensor memory read and region R free for the next chunk
        tc_fence_after();
    }
    if (!ok) {
        // a wait ran out: one more bounded wait for the weight copy and the MMAs in flight
        // before the shared and tensor memory they use are released
        if (tid == 0) {
            raise_status(a.status, ST_TIMEOUT);
            if (!weights_ok) mbar_wait(wbar, 0);
        }
        mbar_wait(bar, (commits - 1) & 1u);
        tc_fence_before();
        __syncthreads();
    } else if (!weights_waited && tid == 0) {
        mbar_wait(wbar, 0);  // a CTA without chunks still lets its weight copy land
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

int32_t tc_ctas_per_sm(int *out) {
    static bool configured = false;
    if (!configured) {
        DDG_CU(cudaFuncSetAttribute(k_dss_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
        configured = true;
    }
    DDG_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_dss_tc, TC_T, TC_SMEM));
    if (*out > TC_CTAS_PER_SM) {
        set_error("schedule 4 needs at most four CTAs per SM");
        return DDG_INTERNAL;
    }
    return DDG_OK;
}

int32_t dss_tc_launch(ddg_problem *p, const ChunkArgs &base, const float *fused_host, const float *tc_w,
                      cudaStream_t s) {
    int per_sm = 0, sms = 0;
    DDG_TRY(tc_ctas_per_sm(&per_sm));
    DDG_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->ctx->device));
    const ddg_model *m = p->model;
    const int nc = p->chunk.nchunks;
    // four CTAs per SM (the shared-memory size allows no more; CTAs beyond the resident ones
    // only start later), each looping over its chunks
    const int grid = std::max(1, std::min(nc, sms * TC_CTAS_PER_SM));
    for (int blk = 0; blk < m->kbar; ++blk) {
        ChunkArgs a = base;
        a.first = blk == 0;
        a.last = blk == m->kbar - 1;
        a.h_in = (blk & 1) ? p->dss_h2 : p->dss_h;
        a.h_out = (blk & 1) ? p->dss_h : p->dss_h2;
        const FusedWeights *Wb = reinterpret_cast<const FusedWeights *>(fused_host) + blk;
        const float *img = tc_w + (size_t)blk * TCW_FLOATS;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(TC_T);
        cfg.dynamicSmemBytes = TC_SMEM;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = p->ctx->pdl ? 1 : 0;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        DDG_CU(cudaLaunchKernelEx(&cfg, k_dss_tc, *Wb, a, img, nc));
    }
    DDG_LAUNCHES(m->kbar);
    return DDG_OK;
}

}  // namespace ddg
