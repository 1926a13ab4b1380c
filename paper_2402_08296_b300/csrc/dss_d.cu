// Schedule 5 of the batched Deep Statistical Solver inference (Section III-B, Eqs. 18-22) for
// latent sizes other than the d = 10 compiled into schedules 0-4: d = 5 and d = 20, the other
// columns of Table 2's (kbar, d) sweep.  One launch per message-passing block over the chunks
// of schedule 2 (each chunk holds at most 2T nodes of one local graph), one thread per own
// node, the weights of the block in shared memory in the flat layout of the model
// (row-major W[out][in], per block: Phi_out, Phi_in, Psi, decoder; 11 d^2 + 15 d + 1 floats).
//
// The edge MLPs are evaluated in factorised form as in schedule 2: with W1 = [Wa | Wb | We],
//   W1 [h_j, h_l, e] + b1 = (Wa h_j + b1) + Wb h_l + We e,
// so phase A stores every needed node's projections Wb_out h and Wb_in h in shared memory and
// phase B forms each edge's hidden pre-activation from them; the second layer is applied once
// to the per-node sum: sum_l (W2 relu(z_jl) + b2) = W2 sum_l relu(z_jl) + deg_j b2.
// Latents live in d planes of sum_loc floats between the launches.
#include "dss_layout.cuh"

namespace ddg {

template <int DD>
struct FlatD {
    static constexpr int IN1 = 2 * DD + 3, INP = 3 * DD + 1;
    static constexpr int PO_W1 = 0, PO_B1 = PO_W1 + DD * IN1, PO_W2 = PO_B1 + DD, PO_B2 = PO_W2 + DD * DD;
    static constexpr int PI_W1 = PO_B2 + DD, PI_B1 = PI_W1 + DD * IN1, PI_W2 = PI_B1 + DD, PI_B2 = PI_W2 + DD * DD;
    static constexpr int PS_W1 = PI_B2 + DD, PS_B1 = PS_W1 + DD * INP, PS_W2 = PS_B1 + DD, PS_B2 = PS_W2 + DD * DD;
    static constexpr int DE_W1 = PS_B2 + DD, DE_B1 = DE_W1 + DD * DD, DE_W2 = DE_B1 + DD, DE_B2 = DE_W2 + DD;
    static constexpr int SIZE = DE_B2 + 1;
    static_assert(SIZE == 11 * DD * DD + 15 * DD + 1, "flat block size (Table 2's weight count)");
};

// y[o] += sum_i W[o * ld + i] x[i] for NIN inputs, W in shared memory (same address on every
// thread of a warp: a broadcast)
template <int NOUT, int NIN>
__device__ __forceinline__ void mv_flat(float (&y)[NOUT], const float *W, int ld, const float *x) {
#pragma unroll
    for (int o = 0; o < NOUT; ++o) {
        float acc = y[o];
#pragma unroll
        for (int i = 0; i < NIN; ++i) acc = fmaf(W[o * ld + i], x[i], acc);
        y[o] = acc;
    }
}

template <int DD, int T>
__global__ void __launch_bounds__(T) k_dss_chunk_d(const __grid_constant__ ChunkArgs a, const float *wblock) {
    using F = FlatD<DD>;
    extern __shared__ __align__(16) float smd[];
    float *Ws = smd;                  // [F::SIZE] weights of the block
    float *Pb = smd + ((F::SIZE + 3) & ~3);  // [needed][2 DD] projections (out, in)
    if (a.stop && *a.stop) return;
    const int q = blockIdx.x, tid = threadIdx.x;
    const int g = a.c_graph[q];
    const int lp = a.loc_ptr[g];
    const int k = a.loc_nint[g];
    const int s0 = a.sub_ptr[g];
    const double s = a.s[g];
    const int n0 = a.c_n0[q], own = a.c_own[q];
    const int nn = a.c_need_n[q];
    const int *need = a.need + a.c_need_off[q];
    if (s == 0.0) {  // zero restricted residual: no correction (the CTA returns as a whole)
        if (a.last)
            for (int t = tid; t < own; t += T)
                if (n0 + t < k) a.corr[s0 + n0 + t] = 0.0;
        return;
    }
    for (int i = tid; i < F::SIZE; i += T) Ws[i] = wblock[i];
    __syncthreads();
    // phase A: projections Wb_out h and Wb_in h of every needed node
    for (int u = tid; u < nn; u += T) {
        const int j = need[u];
        float h[DD], po[DD], pi[DD];
#pragma unroll
        for (int o = 0; o < DD; ++o) {
            h[o] = a.first ? 0.f : a.h_in[(size_t)o * a.n_total + lp + j];
            po[o] = 0.f;
            pi[o] = 0.f;
        }
        mv_flat<DD, DD>(po, Ws + F::PO_W1 + DD, F::IN1, h);
        mv_flat<DD, DD>(pi, Ws + F::PI_W1 + DD, F::IN1, h);
        float *dst = Pb + (size_t)u * 2 * DD;
#pragma unroll
        for (int o = 0; o < DD; ++o) {
            dst[o] = po[o];
            dst[DD + o] = pi[o];
        }
    }
    __syncthreads();
    const int *aptr = a.adj_ptr + a.c_adj_off[q];
    const uint16_t *adj = a.adj + a.c_adj_base[q];
    const float2 *xy = a.loc_xy + lp;
    for (int u = tid; u < own; u += T) {
        const int j = n0 + u;  // graph-local id
        const bool inner = j < k;
        float h[DD], c;
        if (a.first) {
            c = inner ? (float)(a.r[a.sub_idx[s0 + j]] / s) : 0.f;
            a.c[lp + j] = c;
#pragma unroll
            for (int o = 0; o < DD; ++o) h[o] = 0.f;
        } else {
            c = a.c[lp + j];
#pragma unroll
            for (int o = 0; o < DD; ++o) h[o] = a.h_in[(size_t)o * a.n_total + lp + j];
        }
        const float2 xj = xy[j];
        float pao[DD], pai[DD], so[DD], si[DD];
#pragma unroll
        for (int o = 0; o < DD; ++o) {
            pao[o] = Ws[F::PO_B1 + o];
            pai[o] = Ws[F::PI_B1 + o];
            so[o] = 0.f;
            si[o] = 0.f;
        }
        mv_flat<DD, DD>(pao, Ws + F::PO_W1, F::IN1, h);
        mv_flat<DD, DD>(pai, Ws + F::PI_W1, F::IN1, h);
        int dout = 0, din = 0;
        for (int e = aptr[u]; e < aptr[u + 1]; ++e) {
            const int v = adj[e];   // chunk-local
            const int l = need[v];  // graph-local
            const float2 xl = xy[l];
            const float dx = xl.x - xj.x, dy = xl.y - xj.y;
            const float dn = sqrtf(dx * dx + dy * dy);
            const float *pbl = Pb + (size_t)v * 2 * DD;
            if (l < k) {  // out-message to an unknown (Eq. 18, d_jl = x_l - x_j)
#pragma unroll
                for (int o = 0; o < DD; ++o) {
                    const float *we = Ws + F::PO_W1 + o * F::IN1 + 2 * DD;
                    float z = pao[o] + pbl[o];
                    z = fmaf(we[0], dx, z);
                    z = fmaf(we[1], dy, z);
                    z = fmaf(we[2], dn, z);
                    so[o] += relu(z);
                }
                ++dout;
            }
            if (inner) {  // in-message (Eq. 19, d_lj = x_j - x_l)
#pragma unroll
                for (int o = 0; o < DD; ++o) {
                    const float *we = Ws + F::PI_W1 + o * F::IN1 + 2 * DD;
                    float z = pai[o] + pbl[DD + o];
                    z = fmaf(we[0], -dx, z);
                    z = fmaf(we[1], -dy, z);
                    z = fmaf(we[2], dn, z);
                    si[o] += relu(z);
                }
                ++din;
            }
        }
        // second layers on the sums: phi = W2 S + deg b2
        float phi_o[DD], phi_i[DD];
#pragma unroll
        for (int o = 0; o < DD; ++o) {
            phi_o[o] = (float)dout * Ws[F::PO_B2 + o];
            phi_i[o] = (float)din * Ws[F::PI_B2 + o];
        }
        mv_flat<DD, DD>(phi_o, Ws + F::PO_W2, DD, so);
        mv_flat<DD, DD>(phi_i, Ws + F::PI_W2, DD, si);
        // Psi on [h, c, phi_out, phi_in] (Eq. 20), then the ResNet update
        float hid[DD];
#pragma unroll
        for (int o = 0; o < DD; ++o) {
            const float *w = Ws + F::PS_W1 + o * F::INP;
            float acc = Ws[F::PS_B1 + o];
#pragma unroll
            for (int i = 0; i < DD; ++i) acc = fmaf(w[i], h[i], acc);
            acc = fmaf(w[DD], c, acc);
#pragma unroll
            for (int i = 0; i < DD; ++i) acc = fmaf(w[DD + 1 + i], phi_o[i], acc);
#pragma unroll
            for (int i = 0; i < DD; ++i) acc = fmaf(w[2 * DD + 1 + i], phi_i[i], acc);
            hid[o] = relu(acc);
        }
        float out[DD];
#pragma unroll
        for (int o = 0; o < DD; ++o) out[o] = Ws[F::PS_B2 + o];
        mv_flat<DD, DD>(out, Ws + F::PS_W2, DD, hid);
#pragma unroll
        for (int o = 0; o < DD; ++o) h[o] = fmaf(a.alpha, out[o], h[o]);
        if (a.last) {
            if (inner) {  // decoder of the last block (Eq. 22)
                float dh[DD];
#pragma unroll
                for (int o = 0; o < DD; ++o) dh[o] = Ws[F::DE_B1 + o];
                mv_flat<DD, DD>(dh, Ws + F::DE_W1, DD, h);
                float y = Ws[F::DE_B2];
#pragma unroll
                for (int o = 0; o < DD; ++o) y = fmaf(Ws[F::DE_W2 + o], relu(dh[o]), y);
                a.corr[s0 + j] = s * (double)y;
            }
        } else {
#pragma unroll
            for (int o = 0; o < DD; ++o) a.h_out[(size_t)o * a.n_total + lp + j] = h[o];
        }
    }
}

constexpr int DSS_D_T = 128;

template <int DD>
static int32_t launch_d(ddg_problem *p, const ChunkArgs &base, cudaStream_t s) {
    using F = FlatD<DD>;
    static bool configured = false;
    if (!configured) {
        DDG_CU(cudaFuncSetAttribute(k_dss_chunk_d<DD, DSS_D_T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    227 * 1024));
        configured = true;
    }
    const size_t smem = sizeof(float) * ((size_t)((F::SIZE + 3) & ~3) + (size_t)p->chunk.max_need * 2 * DD);
    if (smem > 227 * 1024) {
        set_error("a GNN chunk needs more shared memory than a CTA has");
        return DDG_TOO_LARGE;
    }
    const ddg_model *m = p->model;
    for (int blk = 0; blk < m->kbar; ++blk) {
        ChunkArgs a = base;
        a.first = blk == 0;
        a.last = blk == m->kbar - 1;
        a.h_in = (blk & 1) ? p->dss_h2 : p->dss_h;
        a.h_out = (blk & 1) ? p->dss_h : p->dss_h2;
        k_dss_chunk_d<DD, DSS_D_T><<<p->chunk.nchunks, DSS_D_T, smem, s>>>(a, m->w + (size_t)blk * F::SIZE);
    }
    DDG_LAUNCHES(m->kbar);
    return DDG_OK;
}

int32_t dss_d_launch(ddg_problem *p, const ChunkArgs &a, cudaStream_t s) {
    switch (p->model->d) {
        case 5: return launch_d<5>(p, a, s);
        case 10: return launch_d<10>(p, a, s);
        case 20: return launch_d<20>(p, a, s);
        default: set_error("latent size d must be 5, 10 or 20"); return DDG_INVALID_ARG;
    }
}

}  // namespace ddg
