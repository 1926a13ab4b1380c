// Packed per-block weight layout of the GNN kernels and their shared device helpers.
#pragma once

#include "ddg_internal.cuh"

namespace ddg {

// ---------------------------------------------------------------- packed layout (d = 10, rows padded to 12)
constexpr int D = DSS_D;
constexpr int DP = 12;
// one edge MLP
constexpr int PHI_WA = 0;                 // [D][DP] Wa^T
constexpr int PHI_WB = PHI_WA + D * DP;   // [D][DP] Wb^T
constexpr int PHI_WE = PHI_WB + D * DP;   // [3][DP] We^T
constexpr int PHI_B1 = PHI_WE + 3 * DP;   // [DP]
constexpr int PHI_W2 = PHI_B1 + DP;       // [D][DP] W2^T
constexpr int PHI_B2 = PHI_W2 + D * DP;   // [DP]
constexpr int PHI_SIZE = PHI_B2 + DP;     // 420
// block
constexpr int OFF_OUT = 0;
constexpr int OFF_IN = PHI_SIZE;
constexpr int OFF_PSI = 2 * PHI_SIZE;
constexpr int PSI_W1 = 0;                      // [3D+1][DP]
constexpr int PSI_B1 = PSI_W1 + (3 * D + 1) * DP;
constexpr int PSI_W2 = PSI_B1 + DP;            // [D][DP]
constexpr int PSI_B2 = PSI_W2 + D * DP;
constexpr int PSI_SIZE = PSI_B2 + DP;          // 516
constexpr int OFF_DEC = OFF_PSI + PSI_SIZE;
constexpr int DEC_W1 = 0;                      // [D][DP]
constexpr int DEC_B1 = DEC_W1 + D * DP;
constexpr int DEC_W2 = DEC_B1 + DP;            // [DP]
constexpr int DEC_B2 = DEC_W2 + DP;            // [4]
constexpr int DEC_SIZE = DEC_B2 + 4;           // 148
constexpr int BLOCK_FLOATS = OFF_DEC + DEC_SIZE;  // 1504
constexpr int BLOCK_BYTES = BLOCK_FLOATS * 4;     // 6016, a multiple of 16
static_assert(BLOCK_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");

// ---------------------------------------------------------------- fused layout (schedule 3)
// Per block, every matrix stored input-major ([in][out]) so that consecutive
// outputs form 8-byte pairs for the packed two-lane FP32 instructions:
//   HB  [D][2D]  Wb_out and Wb_in interleaved by output pairs (o0 o1 i0 i1 o2 o3 ...),
//                the layout of a node's neighbour projections in shared memory
//   HA  [D][3D]  Wa_out | Wa_in | the h-columns of Psi's first layer;  BA [3D] their biases
//   WEO [3][D]   We_out for (dx, dy, |d|);  WEI [3][D] We_in for (-dx, -dy, |d|), signs folded in
//   MO, MI [D][D]  Psi_W1(phi_out cols) W2_out and Psi_W1(phi_in cols) W2_in, composed
//   VC [D]       Psi_W1 column of c;  VO, VI [D]  Psi_W1(phi cols) b2 (times the degree)
//   P2 [D][D]    alpha Psi_W2;  PB2 [D]  alpha Psi_b2
//   DW1 [D][D], DB1 [D], DW2 [D], DB2 [2]  decoder
// The compositions are exact in real arithmetic:
//   Psi_W1 [.., phi, ..] with phi = W2 S + deg b2  =  (Psi_W1 W2) S + deg (Psi_W1 b2).
constexpr int F_HB = 0;
constexpr int F_HA = F_HB + D * 2 * D;
constexpr int F_BA = F_HA + D * 3 * D;
constexpr int F_WEO = F_BA + 3 * D;
constexpr int F_WEI = F_WEO + 3 * D;
constexpr int F_MO = F_WEI + 3 * D;
constexpr int F_MI = F_MO + D * D;
constexpr int F_VC = F_MI + D * D;
constexpr int F_VO = F_VC + D;
constexpr int F_VI = F_VO + D;
constexpr int F_P2 = F_VI + D;
constexpr int F_PB2 = F_P2 + D * D;
constexpr int F_DW1 = F_PB2 + D;
constexpr int F_DB1 = F_DW1 + D * D;
constexpr int F_DW2 = F_DB1 + D;
constexpr int F_DB2 = F_DW2 + D;
// the position part of the edge features, moved into per-node terms (schedule 3):
//   We (x_l - x_j) = We x_l - We x_j, so the neighbour projection gains We x_l and the own-node
//   term loses We x_j; only We_|d| |d| stays on the edge.
//   XB  [2][2D]  rows x, y of We_out and We_in interleaved like HB (added to a neighbour's projections)
//   NXA [2][2D]  rows x, y of -We_out | -We_in (added to the own node's first-layer terms)
constexpr int F_XB = F_DB2 + 2;
constexpr int F_NXA = F_XB + 2 * 2 * D;
constexpr int F_FLOATS = F_NXA + 2 * 2 * D;  // 1132
static_assert(F_FLOATS % 2 == 0 && F_HA % 2 == 0 && F_MO % 2 == 0 && F_P2 % 2 == 0 && F_DW1 % 2 == 0 &&
                  F_XB % 2 == 0 && F_NXA % 2 == 0,
              "every pair starts on an 8-byte boundary");

struct alignas(16) FusedWeights {
    float w[F_FLOATS];
};

// ---------------------------------------------------------------- packed two-lane FP32 (f32x2)
typedef unsigned long long f2_t;  // lanes (lo, hi)

__device__ __forceinline__ f2_t f2_pack(float lo, float hi) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
    f2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ReLU as max(x, 0) that keeps a NaN input (max.NaN); fmaxf would return 0 for it
__device__ __forceinline__ float relu(float x) {
    float r;
    asm("max.NaN.f32 %0, %1, 0f00000000;" : "=f"(r) : "f"(x));
    return r;
}

// ---------------------------------------------------------------- bulk copy + mbarrier helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// wait on a phase of an mbarrier for at most about one second; returns false if that ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (globaltimer_ns() - t0 > 1000000000ull) return false;
    }
}

template <int NIN>
__device__ __forceinline__ void mv_acc(float (&acc)[D], const float *WT, const float *x) {
#pragma unroll
    for (int i = 0; i < NIN; ++i) {
        const float4 w0 = *reinterpret_cast<const float4 *>(WT + i * DP);
        const float4 w1 = *reinterpret_cast<const float4 *>(WT + i * DP + 4);
        const float2 w2 = *reinterpret_cast<const float2 *>(WT + i * DP + 8);
        const float xi = x[i];
        acc[0] = fmaf(w0.x, xi, acc[0]);
        acc[1] = fmaf(w0.y, xi, acc[1]);
        acc[2] = fmaf(w0.z, xi, acc[2]);
        acc[3] = fmaf(w0.w, xi, acc[3]);
        acc[4] = fmaf(w1.x, xi, acc[4]);
        acc[5] = fmaf(w1.y, xi, acc[5]);
        acc[6] = fmaf(w1.z, xi, acc[6]);
        acc[7] = fmaf(w1.w, xi, acc[7]);
        acc[8] = fmaf(w2.x, xi, acc[8]);
        acc[9] = fmaf(w2.y, xi, acc[9]);
    }
}

__device__ __forceinline__ void load_vec(float (&v)[D], const float *src) {
#pragma unroll
    for (int o = 0; o < D; ++o) v[o] = src[o];
}

// z = P_a + P_b(l) + We e  ->  S += relu(z)
__device__ __forceinline__ void edge_msg(float (&S)[D], const float (&Pa)[D], const float *Pb, const float *We,
                                         float ex, float ey, float en) {
#pragma unroll
    for (int o = 0; o < D; ++o) {
        float z = Pa[o] + Pb[o];
        z = fmaf(We[o], ex, z);
        z = fmaf(We[DP + o], ey, z);
        z = fmaf(We[2 * DP + o], en, z);
        S[o] += relu(z);
    }
}

__device__ __forceinline__ f2_t f2_relu(f2_t v) {
    float lo, hi;
    f2_unpack(v, lo, hi);
    return f2_pack(relu(lo), relu(hi));
}

// max(q, -a) lane by lane; a NaN in either stays NaN (max.NaN)
__device__ __forceinline__ f2_t f2_max_neg(f2_t q, f2_t a) {
    float q0, q1, a0, a1, r0, r1;
    f2_unpack(q, q0, q1);
    f2_unpack(a, a0, a1);
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r0) : "f"(q0), "f"(-a0));
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r1) : "f"(q1), "f"(-a1));
    return f2_pack(r0, r1);
}

// square root by the hardware approximation (relative error near one ulp)
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}


// ---------------------------------------------------------------- chunked schedules (2, 3, 4)
struct ChunkArgs {
    const int *c_graph, *c_n0, *c_own;      // per chunk: graph, first own node (graph-local), own count
    const int *c_need_off, *c_need_n;       // per chunk: start / count of its needed-node list
    const int *need;                        // graph-local ids: own nodes first, then outside neighbours
    const int *c_adj_off;                   // per chunk: start of its own nodes' CSR in adj_ptr
    const int *adj_ptr;                     // own-node CSR offsets (relative to the chunk's adj start)
    const uint16_t *adj;                    // chunk-local neighbour ids
    const uint2 *adjx;                      // schedule 4: {chunk-local neighbour id, |d| float bits}, unknowns first
    const int *c_adj_base;                  // per chunk: start of its slice in adj
    const int *loc_ptr, *loc_nint, *sub_ptr, *sub_idx;
    const int *gid;                         // global plans: graph of every local node
    const int4 *info;                       // global plans: per own slot {node, corr idx, r idx, graph | dout << 24}
    const float2 *loc_xy;
    const double *r, *s;
    double *corr;
    const float *h_in;                      // [D][n_total]
    float *h_out;                           // [D][n_total]
    float *c;                               // [n_total]
    long long n_total;
    float alpha;
    int first, last;
    const int *stop;
    int *status;                            // device status word (bits ST_*)
};

// h (10 floats) and c of a local node from its 12-float latent row
__device__ __forceinline__ void load_hrow(const float4 *rows, int node, float (&h)[D], float &c) {
    const float4 r0 = rows[3 * (size_t)node], r1 = rows[3 * (size_t)node + 1], r2 = rows[3 * (size_t)node + 2];
    h[0] = r0.x; h[1] = r0.y; h[2] = r0.z; h[3] = r0.w;
    h[4] = r1.x; h[5] = r1.y; h[6] = r1.z; h[7] = r1.w;
    h[8] = r2.x; h[9] = r2.y;
    c = r2.z;
}

// acc[m] += sum_i W[OFF + i*STRIDE + 2m .. 2m+1] x_i  over i < D (pairs of outputs)
template <int OFF, int STRIDE>
__device__ __forceinline__ void f2_mv(f2_t (&acc)[D / 2], const f2_t *Wp, const float (&x)[D]) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const f2_t xi = f2_pack(x[i], x[i]);
#pragma unroll
        for (int m = 0; m < D / 2; ++m) acc[m] = f2_fma(Wp[(OFF + i * STRIDE) / 2 + m], xi, acc[m]);
    }
}

// one message pair-block with the position terms already in pa and pb:
// acc += mask * relu(pa + pb + We_|d| |d|)
template <int OFF_WE, bool MASKED>
__device__ __forceinline__ void f2_msg_n(f2_t (&acc)[D / 2], const f2_t (&pa)[D / 2], const f2_t (&pb)[D / 2],
                                         const f2_t *Wp, f2_t dn2, f2_t mask2) {
#pragma unroll
    for (int m = 0; m < D / 2; ++m) {
        f2_t z = f2_add(pa[m], pb[m]);
        z = f2_fma(Wp[(OFF_WE + 2 * D) / 2 + m], dn2, z);
        acc[m] = MASKED ? f2_fma(f2_relu(z), mask2, acc[m]) : f2_add(acc[m], f2_relu(z));
    }
}

}  // namespace ddg
