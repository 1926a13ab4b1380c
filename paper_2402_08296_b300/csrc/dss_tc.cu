// Schedule 4 of the batched Deep Statistical Solver inference (Section III-B, Eqs. 18-22):
// chunks of the concatenated local graphs as in schedule 3 (one launch per message-passing
// block), with the per-node matrix products that take a node's latent vector as input on the
// fifth-generation tensor cores, and the edge messages and the rest of Psi on the CUDA cores.
//
// Per block, a CTA of 128 threads runs one chunk of at most 128 own nodes (one thread per own
// node) and 256 needed nodes (own nodes first, then their neighbours outside the chunk):
//   GEMM (tensor cores, every needed node): [h, x, y, c, d_out, d_in, 1] (16 inputs) -> 64
//     outputs: the neighbour projections Wb h + We_xy x of both edge MLPs (Eqs. 18-19, in the
//     interleaved order the edge loop reads from shared memory), and for own nodes the
//     first-layer terms Wa h + b1 - We_xy x_j of both messages and the h, c and degree part of
//     Psi's hidden layer (Eq. 20, with the message MLPs' second layers composed into it);
//   edge loop (CUDA cores): S_out, S_in = sums over the neighbours of relu(pa + pb + We_|d| |d|);
//   Psi (CUDA cores): hidden = GEMM part + (Psi_W1 W2)[S_out, S_in], then h += alpha (Psi_W2
//     relu(hidden) + Psi_b2); the decoder (Eq. 22) of the last block.
// The GEMM is one tcgen05.mma chain (kind::tf32) per 128-row tile, issued by one thread from
// shared-memory operands into FP32 accumulators in tensor memory, read back with tcgen05.ld,
// whose 32x32b shape hands every thread the row of the node it owns.  FP32 accuracy from the
// TF32 tensor cores by a three-term split: the tensor core truncates its FP32 inputs to TF32,
// so x W = x W_hi + x_lo W_hi + x W_lo up to terms below 2^-20 relative, with W_hi = W
// truncated to TF32 and W_lo = W - W_hi (both exact in FP32) and x_lo = x - trunc(x), each
// product one more K-concatenated term of the same accumulator.
//
// Operands are K-major without swizzling: 8-row x 16-byte core matrices, the K-chunks of a
// row group contiguous (leading-dimension byte offset 128 between core matrices along K,
// stride-dimension byte offset K/4 * 128 between row groups).  The weights of the block come
// with one bulk copy.  Tensor memory: 128 columns per CTA (tile 0 at column 0, N = 64; tile 1,
// which holds outside neighbours only, at column 64, N = 32), freed as soon as the results are
// read; the CTA's shared memory keeps at most four CTAs on an SM, so the 512 columns of an SM
// always suffice and an allocation never waits.  Every wait on a barrier is bounded (about one
// second), after which the CTA raises ST_TIMEOUT, waits once more, frees its tensor memory and
// returns.
#include "dss_layout.cuh"

#include <cstring>

namespace ddg {

// ---------------------------------------------------------------- weight image of one block
constexpr int TC_KA = 16, TC_NA = 64;
static_assert(2 * TC_NA * TC_KA == TCW_FLOATS, "weight image size");
static_assert((TCW_FLOATS * 4) % 16 == 0, "the image is one bulk copy of whole 16-byte pieces");

// shared memory of a CTA (bytes): the GEMM's operand rows (X and its low part XL), overlaid after
// the GEMM by the neighbour projections; the weight image; scaled coordinates; barriers and the
// tensor-memory address
constexpr int TC_OFF_XL = TC_NEED * TC_KA * 4;        // 16384
constexpr int TC_OFF_W = 2 * TC_OFF_XL;               // 32768
constexpr int TC_OFF_XY = TC_OFF_W + TCW_FLOATS * 4;  // 40960
constexpr int TC_OFF_BAR = TC_OFF_XY + TC_NEED * 8;   // 43008: MMA barrier, weight barrier, TMEM address
static_assert(TC_NEED * 80 <= TC_OFF_W, "the projections fit over the operand rows");
static_assert(TC_OFF_BAR + 24 <= (int)TC_SMEM, "shared memory layout");
static_assert(5 * TC_SMEM > 228 * 1024, "at most four schedule-4 CTAs per SM (4 x 128 TMEM columns)");

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

static void put_w(float *img, int r, int k, float w) {
    const float hi = tf32_high(w);
    img[tc_core(r, k, TC_KA)] = hi;
    img[TC_NA * TC_KA + tc_core(r, k, TC_KA)] = w - hi;
}

// The B operand of every block, from the composed per-block layout of schedule 3
// (dss_layout.cuh): row = output, column = input (0-9 h, 10 x, 11 y, 12 c, 13 d_out, 14 d_in,
// 15 one).  Rows 0-19 the projections, out/in pairs interleaved as in shared memory; 20-29
// pa_out; 30-39 pa_in; 40-49 the GEMM's part of Psi's hidden layer; 50-63 zero.
void tc_weight_image(const float *fused, int kbar, std::vector<float> &img) {
    img.assign((size_t)kbar * TCW_FLOATS, 0.f);
    for (int b = 0; b < kbar; ++b) {
        const float *f = fused + (size_t)b * F_FLOATS;
        float *o = img.data() + (size_t)b * TCW_FLOATS;
        for (int r = 0; r < 2 * D; ++r) {
            for (int i = 0; i < D; ++i) put_w(o, r, i, f[F_HB + i * 2 * D + r]);
            put_w(o, r, 10, f[F_XB + r]);
            put_w(o, r, 11, f[F_XB + 2 * D + r]);
        }
        for (int q = 0; q < D; ++q) {
            const int ro = 2 * D + q, ri = 3 * D + q, rh = 4 * D + q;
            for (int i = 0; i < D; ++i) {
                put_w(o, ro, i, f[F_HA + i * 3 * D + q]);
                put_w(o, ri, i, f[F_HA + i * 3 * D + D + q]);
                put_w(o, rh, i, f[F_HA + i * 3 * D + 2 * D + q]);
            }
            put_w(o, ro, 10, f[F_NXA + q]);
            put_w(o, ro, 11, f[F_NXA + 2 * D + q]);
            put_w(o, ro, 15, f[F_BA + q]);
            put_w(o, ri, 10, f[F_NXA + D + q]);
            put_w(o, ri, 11, f[F_NXA + 3 * D + q]);
            put_w(o, ri, 15, f[F_BA + D + q]);
            put_w(o, rh, 12, f[F_VC + q]);
            put_w(o, rh, 13, f[F_VO + q]);
            put_w(o, rh, 14, f[F_VI + q]);
            put_w(o, rh, 15, f[F_BA + 2 * D + q]);
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
// a descriptor's address field by 2 core matrices = 256 bytes = 16 units)
__device__ __forceinline__ void tc_gemm3(uint32_t d, uint64_t ax, uint64_t axl, uint64_t bh, uint64_t bl, int steps,
                                         uint32_t idesc) {
    int acc = 0;
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

// ---------------------------------------------------------------- the kernel
__global__ void __launch_bounds__(TC_T, 4)
    k_dss_tc(const __grid_constant__ FusedWeights W, const __grid_constant__ ChunkArgs a, const float *wimg) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    if (a.stop && *a.stop) return;
    float *X = reinterpret_cast<float *>(tsm);
    float *XL = reinterpret_cast<float *>(tsm + TC_OFF_XL);
    float4 *Pb = reinterpret_cast<float4 *>(tsm);  // over the operand rows once the GEMM is done
    float *Ws = reinterpret_cast<float *>(tsm + TC_OFF_W);
    float2 *XY = reinterpret_cast<float2 *>(tsm + TC_OFF_XY);
    uint64_t *bar = reinterpret_cast<uint64_t *>(tsm + TC_OFF_BAR);
    uint64_t *wbar = bar + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tsm + TC_OFF_BAR + 16);
    const int q = blockIdx.x, tid = threadIdx.x, warp = tid >> 5;
    const int own = a.c_own[q];
    const int nn = a.c_need_n[q];
    const int *need = a.need + a.c_need_off[q];
    const int *APTR = a.adj_ptr + a.c_adj_off[q];
    const uint16_t *ADJ = a.adj + a.c_adj_base[q];
    const int4 *INFO = a.info + a.c_n0[q];
    const f2_t *Wp = reinterpret_cast<const f2_t *>(W.w);
    const float4 *hrow_in = reinterpret_cast<const float4 *>(a.h_in);
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
    asm volatile("griddepcontrol.wait;" ::: "memory");

    // ---- GEMM operand rows: row tid (tile 0) and row 128 + tid (tile 1, outside neighbours)
    float h[D], c = 0.f;
    int4 inf = make_int4(0, -1, 0, 0);
    bool inner = false;
#pragma unroll
    for (int o = 0; o < D; ++o) h[o] = 0.f;
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const int u = tid + rr * TC_T;
        if (u >= nn) continue;
        const int node = need[u];
        const float2 xy = a.loc_xy[node];
        float v[TC_KA], cv = 0.f;
#pragma unroll
        for (int o = 0; o < TC_KA; ++o) v[o] = 0.f;
        if (!first) {
            float hv[D];
            load_hrow(hrow_in, node, hv, cv);
#pragma unroll
            for (int o = 0; o < D; ++o) v[o] = hv[o];
        }
        v[10] = xy.x;
        v[11] = xy.y;
        if (u < own) {  // rr == 0: the own node of this thread
            inf = INFO[u];
            inner = inf.y >= 0;
            if (first) {
                const double s = a.s[inf.w & 0xffffff];
                cv = (inner && s != 0.0) ? (float)(a.r[inf.z] / s) : 0.f;
            }
            v[12] = cv;
            v[13] = (float)((unsigned)inf.w >> 24);
            v[14] = inner ? (float)(APTR[u + 1] - APTR[u]) : 0.f;
            v[15] = 1.f;
#pragma unroll
            for (int o = 0; o < D; ++o) h[o] = v[o];
            c = cv;
        }
        tc_put_row<TC_KA>(X, XL, u, v);
        XY[u] = xy;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
    bool ok = true;
    if (warp == 0) {
        if (tid == 0) {
            ok = mbar_wait(wbar, 0);
            if (ok) {
                tc_fence_after();
                const uint64_t bh = tc_desc(Ws, TC_KA), bl = tc_desc(Ws + TC_NA * TC_KA, TC_KA);
                tc_gemm3(tmem, tc_desc(X, TC_KA), tc_desc(XL, TC_KA), bh, bl, TC_KA / 8, tc_idesc(TC_NA));
                if (nn > TC_T)
                    tc_gemm3(tmem + 64u, tc_desc(X + 128 * TC_KA, TC_KA), tc_desc(XL + 128 * TC_KA, TC_KA), bh, bl,
                             TC_KA / 8, tc_idesc(32));
                tc_commit(bar);
            }
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (ok) ok = mbar_wait(bar, 0);
    }
    // one barrier: warp 0 saw the MMAs complete (or gave up); then every thread observes the
    // completed phase itself before reading tensor memory
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            raise_status(a.status, ST_TIMEOUT);
            mbar_wait(wbar, 0);  // once more for the weight copy in flight into this CTA's shared memory
        }
        mbar_wait(bar, 0);  // and for MMAs in flight before the tensor memory is freed
        tc_fence_before();
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        return;
    }
    mbar_wait(bar, 0);
    tc_fence_after();
    // ---- read back: projections of the needed rows into shared memory (over the operand rows,
    // which the completed GEMM no longer reads); the own node's terms into registers
    f2_t pao[D / 2], pai[D / 2];
    float hp[D];
    {
        float pv[16], pw[4], v0[16], v1[16];
        tmem_ld16(tmem + lane, pv);
        tmem_ld4(tmem + lane + 16, pw);
        tmem_ld16(tmem + lane + 20, v0);  // columns 20-35: pa_out[10], pa_in[0..5]
        tmem_ld16(tmem + lane + 36, v1);  // columns 36-51: pa_in[6..9], hidden part[10], 2 zero
        tmem_wait();
        if (tid < nn) {
#pragma unroll
            for (int m = 0; m < 4; ++m)
                Pb[(size_t)tid * 5 + m] = make_float4(pv[4 * m], pv[4 * m + 1], pv[4 * m + 2], pv[4 * m + 3]);
            Pb[(size_t)tid * 5 + 4] = make_float4(pw[0], pw[1], pw[2], pw[3]);
        }
#pragma unroll
        for (int m = 0; m < D / 2; ++m) pao[m] = f2_pack(v0[2 * m], v0[2 * m + 1]);
        pai[0] = f2_pack(v0[10], v0[11]);
        pai[1] = f2_pack(v0[12], v0[13]);
        pai[2] = f2_pack(v0[14], v0[15]);
        pai[3] = f2_pack(v1[0], v1[1]);
        pai[4] = f2_pack(v1[2], v1[3]);
#pragma unroll
        for (int o = 0; o < D; ++o) hp[o] = v1[4 + o];
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
    // projections complete, tensor memory read: free it for the next CTA on this SM
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    if (tid < own) {
        // ---- edge messages of the own node
        f2_t so[D / 2], si[D / 2];
#pragma unroll
        for (int m = 0; m < D / 2; ++m) so[m] = si[m] = 0ull;
        const float2 xj = XY[tid];
        const int e0 = APTR[tid], e1 = APTR[tid + 1];
        unsigned ent_next = e0 < e1 ? ADJ[e0] : 0u;
        for (int e = e0; e < e1; ++e) {
            const unsigned ent = ent_next;
            if (e + 1 < e1) ent_next = ADJ[e + 1];
            const int v = ent & 0x7fffu;
            const float mo = (float)(ent >> 15);
            const float2 xl = XY[v];
            const float dx = xl.x - xj.x, dy = xl.y - xj.y;
            const float dn = sqrt_approx(fmaf(dx, dx, dy * dy));
            const f2_t dn2 = f2_pack(dn, dn);
            f2_t po[D / 2], pi[D / 2];
#pragma unroll
            for (int m = 0; m < D / 2; ++m) {
                const float4 t = Pb[(size_t)v * 5 + m];
                po[m] = f2_pack(t.x, t.y);
                pi[m] = f2_pack(t.z, t.w);
            }
            f2_msg_n<F_WEO, true>(so, pao, po, Wp, dn2, f2_pack(mo, mo));
            if (inner) f2_msg_n<F_WEI, false>(si, pai, pi, Wp, dn2, 0ull);
        }
        // ---- Psi: hidden = GEMM part + (Psi_W1 W2) [S_out, S_in]; h += alpha (Psi_W2 relu + Psi_b2)
        f2_t hid[D / 2];
#pragma unroll
        for (int m = 0; m < D / 2; ++m) hid[m] = f2_pack(hp[2 * m], hp[2 * m + 1]);
        {
            float sov[D], siv[D];
#pragma unroll
            for (int m = 0; m < D / 2; ++m) {
                f2_unpack(so[m], sov[2 * m], sov[2 * m + 1]);
                f2_unpack(si[m], siv[2 * m], siv[2 * m + 1]);
            }
            f2_mv<F_MO, D>(hid, Wp, sov);
            if (inner) f2_mv<F_MI, D>(hid, Wp, siv);
        }
        f2_t out[D / 2];
        {
            float rh[D];
#pragma unroll
            for (int m = 0; m < D / 2; ++m) {
                float r0, r1;
                f2_unpack(hid[m], r0, r1);
                rh[2 * m] = relu(r0);
                rh[2 * m + 1] = relu(r1);
                out[m] = Wp[F_PB2 / 2 + m];
            }
            f2_mv<F_P2, D>(out, Wp, rh);
        }
        float hn[D];
#pragma unroll
        for (int m = 0; m < D / 2; ++m) {
            const f2_t hv = f2_add(f2_pack(h[2 * m], h[2 * m + 1]), out[m]);
            f2_unpack(hv, hn[2 * m], hn[2 * m + 1]);
        }
        if (last) {
            if (inner) {
                f2_t dh[D / 2];
#pragma unroll
                for (int m = 0; m < D / 2; ++m) dh[m] = Wp[F_DB1 / 2 + m];
                f2_mv<F_DW1, D>(dh, Wp, hn);
                float y = W.w[F_DB2];
#pragma unroll
                for (int m = 0; m < D / 2; ++m) {
                    float d0, d1;
                    f2_unpack(dh[m], d0, d1);
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
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

int32_t tc_ctas_per_sm(int *out) {
    static bool configured = false;
    if (!configured) {
        DDG_CU(cudaFuncSetAttribute(k_dss_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
        configured = true;
    }
    DDG_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_dss_tc, TC_T, TC_SMEM));
    if (*out > 4) {
        set_error("schedule 4 needs at most four CTAs per SM");
        return DDG_INTERNAL;
    }
    return DDG_OK;
}

int32_t dss_tc_launch(ddg_problem *p, const ChunkArgs &base, const float *fused_host, const float *tc_w,
                      cudaStream_t s) {
    int per_sm = 0;
    DDG_TRY(tc_ctas_per_sm(&per_sm));
    const ddg_model *m = p->model;
    for (int blk = 0; blk < m->kbar; ++blk) {
        ChunkArgs a = base;
        a.first = blk == 0;
        a.last = blk == m->kbar - 1;
        a.h_in = (blk & 1) ? p->dss_h2 : p->dss_h;
        a.h_out = (blk & 1) ? p->dss_h : p->dss_h2;
        const FusedWeights *Wb = reinterpret_cast<const FusedWeights *>(fused_host) + blk;
        const float *img = tc_w + (size_t)blk * TCW_FLOATS;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(p->chunk.nchunks);
        cfg.blockDim = dim3(TC_T);
        cfg.dynamicSmemBytes = TC_SMEM;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = p->ctx->pdl ? 1 : 0;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        DDG_CU(cudaLaunchKernelEx(&cfg, k_dss_tc, *Wb, a, img));
    }
    DDG_LAUNCHES(m->kbar);
    return DDG_OK;
}

}  // namespace ddg
