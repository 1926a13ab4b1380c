// Batched Deep Statistical Solver inference (Section III-B, Eqs. 18-22) for all
// subdomain graphs of a decomposition in one launch (Section III-A, Eq. 14).
//
// One CTA runs one local graph through all kbar blocks; graphs are handed out
// largest first.  Each thread owns up to P nodes for the whole inference and
// keeps their latent vectors h (d = 10) and normalised residual c in registers.
// The edge MLPs are evaluated in factorised form: with W1 = [Wa | Wb | We],
//   W1 [h_j, h_l, e] + b1 = (Wa h_j + b1) + (Wb h_l) + We e,
// so phase A of a block stores the per-node projections Wb_out h and Wb_in h
// of every node in shared memory, and phase B forms every edge's hidden
// pre-activation from the owner's Wa h_j + b1, the neighbour's stored
// projection and the 3-vector edge feature; the second layer is applied once
// to the per-node sum: sum_l (W2 relu(z_jl) + b2) = W2 sum_l relu(z_jl) + deg_j b2.
// Edge features: d_jl = x_l - x_j scaled by h_bar for the out-message of j,
// d_lj = x_j - x_l for its in-message, and the Euclidean norm.
// Weights of the next block are fetched with a bulk tensor-memory-access copy
// into the other half of a double buffer while the current block computes.
#include "dss_layout.cuh"

#include <climits>
#include <cstdlib>
#include <cstring>

#include <cmath>

namespace ddg {

// flat layout offsets (row-major W[out][in]) of one block
struct FlatOffsets {
    int phi[2][4];  // W1, b1, W2, b2
    int psi[4];
    int dec[4];
    int size;
};

static FlatOffsets flat_offsets(int d) {
    FlatOffsets f{};
    int o = 0;
    for (int m = 0; m < 2; ++m) {
        f.phi[m][0] = o; o += d * (2 * d + 3);
        f.phi[m][1] = o; o += d;
        f.phi[m][2] = o; o += d * d;
        f.phi[m][3] = o; o += d;
    }
    f.psi[0] = o; o += d * (3 * d + 1);
    f.psi[1] = o; o += d;
    f.psi[2] = o; o += d * d;
    f.psi[3] = o; o += d;
    f.dec[0] = o; o += d * d;
    f.dec[1] = o; o += d;
    f.dec[2] = o; o += d;
    f.dec[3] = o; o += 1;
    f.size = o;
    return f;
}

// one block of the fused layout (see dss_layout.cuh) from one block of flat weights;
// compositions are formed in FP64 and rounded once
static void fuse_block(const float *w, const FlatOffsets &fo, float alpha, float *o) {
    const int in1 = 2 * D + 3, inp = 3 * D + 1;
    const float *Wo1 = w + fo.phi[0][0], *bo1 = w + fo.phi[0][1], *Wo2 = w + fo.phi[0][2], *bo2 = w + fo.phi[0][3];
    const float *Wi1 = w + fo.phi[1][0], *bi1 = w + fo.phi[1][1], *Wi2 = w + fo.phi[1][2], *bi2 = w + fo.phi[1][3];
    const float *P1 = w + fo.psi[0], *pb1 = w + fo.psi[1], *P2 = w + fo.psi[2], *pb2 = w + fo.psi[3];
    const float *dW1 = w + fo.dec[0], *db1 = w + fo.dec[1], *dW2 = w + fo.dec[2], *db2 = w + fo.dec[3];
    for (int i = 0; i < D; ++i)
        for (int m = 0; m < D / 2; ++m)
            for (int t = 0; t < 4; ++t)
                o[F_HB + i * 2 * D + 4 * m + t] =
                    t < 2 ? Wo1[(2 * m + t) * in1 + D + i] : Wi1[(2 * m + t - 2) * in1 + D + i];
    for (int i = 0; i < D; ++i)
        for (int q = 0; q < D; ++q) {
            o[F_HA + i * 3 * D + q] = Wo1[q * in1 + i];
            o[F_HA + i * 3 * D + D + q] = Wi1[q * in1 + i];
            o[F_HA + i * 3 * D + 2 * D + q] = P1[q * inp + i];
        }
    for (int q = 0; q < D; ++q) {
        o[F_BA + q] = bo1[q];
        o[F_BA + D + q] = bi1[q];
        o[F_BA + 2 * D + q] = pb1[q];
        for (int c = 0; c < 3; ++c) {
            o[F_WEO + c * D + q] = Wo1[q * in1 + 2 * D + c];
            o[F_WEI + c * D + q] = (c < 2 ? -1.f : 1.f) * Wi1[q * in1 + 2 * D + c];
        }
        o[F_VC + q] = P1[q * inp + D];
        double vo = 0.0, vi = 0.0;
        for (int t = 0; t < D; ++t) {
            vo += (double)P1[q * inp + D + 1 + t] * bo2[t];
            vi += (double)P1[q * inp + 2 * D + 1 + t] * bi2[t];
        }
        o[F_VO + q] = (float)vo;
        o[F_VI + q] = (float)vi;
        for (int mi = 0; mi < D; ++mi) {
            double so = 0.0, si = 0.0;
            for (int t = 0; t < D; ++t) {
                so += (double)P1[q * inp + D + 1 + t] * Wo2[t * D + mi];
                si += (double)P1[q * inp + 2 * D + 1 + t] * Wi2[t * D + mi];
            }
            o[F_MO + mi * D + q] = (float)so;
            o[F_MI + mi * D + q] = (float)si;
            o[F_P2 + mi * D + q] = (float)((double)alpha * P2[q * D + mi]);
            o[F_DW1 + mi * D + q] = dW1[q * D + mi];
        }
        o[F_PB2 + q] = (float)((double)alpha * pb2[q]);
        o[F_DB1 + q] = db1[q];
        o[F_DW2 + q] = dW2[q];
    }
    o[F_DB2] = db2[0];
    o[F_DB2 + 1] = 0.f;
    // position rows (x, y) of the two edge MLPs' We, with the in-message's sign folded as in WEI
    for (int c = 0; c < 2; ++c)
        for (int m = 0; m < D / 2; ++m)
            for (int t = 0; t < 4; ++t)
                o[F_XB + c * 2 * D + 4 * m + t] = t < 2 ? o[F_WEO + c * D + 2 * m + t] : o[F_WEI + c * D + 2 * m + t - 2];
    for (int c = 0; c < 2; ++c)
        for (int q = 0; q < D; ++q) {
            o[F_NXA + c * 2 * D + q] = -o[F_WEO + c * D + q];
            o[F_NXA + c * 2 * D + D + q] = -o[F_WEI + c * D + q];
        }
}

// both host layouts (padded per-block, composed per-block) from flat weights
static void host_layouts(const std::vector<float> &flat, int kbar, int d, float alpha, std::vector<float> &pk,
                         std::vector<float> &fused) {
    FlatOffsets fo = flat_offsets(d);
    pk.assign((size_t)kbar * BLOCK_FLOATS, 0.f);
    fused.assign((size_t)kbar * F_FLOATS, 0.f);
    for (int k = 0; k < kbar; ++k) {
        const float *w = flat.data() + (size_t)k * fo.size;
        fuse_block(w, fo, alpha, fused.data() + (size_t)k * F_FLOATS);
        float *o = pk.data() + (size_t)k * BLOCK_FLOATS;
        for (int mm = 0; mm < 2; ++mm) {
            float *ph = o + (mm == 0 ? OFF_OUT : OFF_IN);
            const float *W1 = w + fo.phi[mm][0], *b1 = w + fo.phi[mm][1], *W2 = w + fo.phi[mm][2],
                        *b2 = w + fo.phi[mm][3];
            const int in1 = 2 * D + 3;
            for (int oo = 0; oo < D; ++oo) {
                for (int i = 0; i < D; ++i) {
                    ph[PHI_WA + i * DP + oo] = W1[oo * in1 + i];
                    ph[PHI_WB + i * DP + oo] = W1[oo * in1 + D + i];
                    ph[PHI_W2 + i * DP + oo] = W2[oo * D + i];
                }
                for (int i = 0; i < 3; ++i) ph[PHI_WE + i * DP + oo] = W1[oo * in1 + 2 * D + i];
                ph[PHI_B1 + oo] = b1[oo];
                ph[PHI_B2 + oo] = b2[oo];
            }
        }
        float *ps = o + OFF_PSI;
        const float *W1 = w + fo.psi[0], *b1 = w + fo.psi[1], *W2 = w + fo.psi[2], *b2 = w + fo.psi[3];
        for (int oo = 0; oo < D; ++oo) {
            for (int i = 0; i < 3 * D + 1; ++i) ps[PSI_W1 + i * DP + oo] = W1[oo * (3 * D + 1) + i];
            for (int i = 0; i < D; ++i) ps[PSI_W2 + i * DP + oo] = W2[oo * D + i];
            ps[PSI_B1 + oo] = b1[oo];
            ps[PSI_B2 + oo] = b2[oo];
        }
        float *de = o + OFF_DEC;
        const float *dW1 = w + fo.dec[0], *db1 = w + fo.dec[1], *dW2 = w + fo.dec[2], *db2 = w + fo.dec[3];
        for (int oo = 0; oo < D; ++oo) {
            for (int i = 0; i < D; ++i) de[DEC_W1 + i * DP + oo] = dW1[oo * D + i];
            de[DEC_B1 + oo] = db1[oo];
            de[DEC_W2 + oo] = dW2[oo];
        }
        de[DEC_B2] = db2[0];
    }
}

int32_t model_host_layouts(ddg_model *m) {
    std::vector<float> flat(m->n_w);
    DDG_CU(cudaMemcpy(flat.data(), m->w, sizeof(float) * m->n_w, cudaMemcpyDeviceToHost));
    host_layouts(flat, m->kbar, m->d, m->alpha, m->packed_host, m->fused_host);
    // schedule 4's weight images, rebuilt with the layouts so that retrained weights are seen
    std::vector<float> img;
    tc_weight_image(m->fused_host.data(), m->kbar, img);
    if (!m->tc_w) DDG_TRY(dalloc(m->ctx, m->allocs, &m->tc_w, img.size()));
    DDG_CU(cudaMemcpy(m->tc_w, img.data(), sizeof(float) * img.size(), cudaMemcpyHostToDevice));
    mma_weight_image(m->fused_host.data(), m->kbar, img);
    if (!m->mma_w) DDG_TRY(dalloc(m->ctx, m->allocs, &m->mma_w, img.size()));
    DDG_CU(cudaMemcpy(m->mma_w, img.data(), sizeof(float) * img.size(), cudaMemcpyHostToDevice));
    return DDG_OK;
}

int32_t model_pack(ddg_model *m) {
    DDG_TRY(model_host_layouts(m));
    DDG_TRY(dalloc(m->ctx, m->allocs, &m->packed, m->packed_host.size()));
    DDG_CU(cudaMemcpy(m->packed, m->packed_host.data(), sizeof(float) * m->packed_host.size(),
                      cudaMemcpyHostToDevice));
    m->packed_per_block = BLOCK_FLOATS;
    return DDG_OK;
}

// round to the nearest bfloat16, ties to even (NaN stays NaN)
static float round_bf16(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    if ((b & 0x7f800000u) == 0x7f800000u && (b & 0x007fffffu)) return x;
    b = (b + 0x7fffu + ((b >> 16) & 1u)) & 0xffff0000u;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

// the weights a problem's GNN launches read (resolved at launch, so retraining the model is seen)
static const float *w_packed_dev(const ddg_problem *p) { return p->w_bf16 ? p->bf16_packed_dev : p->model->packed; }
static const float *w_packed_host(const ddg_problem *p) {
    return p->w_bf16 ? p->bf16_packed_host.data() : p->model->packed_host.data();
}
static const float *w_fused_host(const ddg_problem *p) {
    return p->w_bf16 ? p->bf16_fused_host.data() : p->model->fused_host.data();
}

int32_t dss_select_weights(ddg_problem *p, bool bf16) {
    const ddg_model *m = p->model;
    p->w_bf16 = bf16;
    p->bf16_packed_dev = nullptr;
    p->bf16_tc_dev = nullptr;
    p->bf16_mma_dev = nullptr;
    if (!bf16) return DDG_OK;
    if (m->d != DSS_D) {
        set_error("BF16 weights need d = 10");
        return DDG_INVALID_ARG;
    }
    std::vector<float> flat(m->n_w);
    DDG_CU(cudaMemcpy(flat.data(), m->w, sizeof(float) * m->n_w, cudaMemcpyDeviceToHost));
    for (float &x : flat) x = round_bf16(x);
    host_layouts(flat, m->kbar, m->d, m->alpha, p->bf16_packed_host, p->bf16_fused_host);
    float *dev = nullptr;
    DDG_TRY(dalloc(p->ctx, p->a_pre, &dev, p->bf16_packed_host.size()));
    DDG_CU(cudaMemcpy(dev, p->bf16_packed_host.data(), sizeof(float) * p->bf16_packed_host.size(),
                      cudaMemcpyHostToDevice));
    p->bf16_packed_dev = dev;
    std::vector<float> img;
    tc_weight_image(p->bf16_fused_host.data(), m->kbar, img);
    float *tdev = nullptr;
    DDG_TRY(dalloc(p->ctx, p->a_pre, &tdev, img.size()));
    DDG_CU(cudaMemcpy(tdev, img.data(), sizeof(float) * img.size(), cudaMemcpyHostToDevice));
    p->bf16_tc_dev = tdev;
    mma_weight_image(p->bf16_fused_host.data(), m->kbar, img);
    float *mdev = nullptr;
    DDG_TRY(dalloc(p->ctx, p->a_pre, &mdev, img.size()));
    DDG_CU(cudaMemcpy(mdev, img.data(), sizeof(float) * img.size(), cudaMemcpyHostToDevice));
    p->bf16_mma_dev = mdev;
    return DDG_OK;
}

// ---------------------------------------------------------------- SplitMix64 Xavier initialisation
__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// value i of stream (seed, tag 2): Xavier-uniform for matrix entries, 0 for biases
__global__ void k_xavier(float *w, int kbar, int d, uint64_t seed, const int *kind, const double *bound, int per_block) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)kbar * per_block) return;
    int q = (int)(i % per_block);
    if (!kind[q]) {
        w[i] = 0.f;
        return;
    }
    uint64_t key = splitmix_mix(seed ^ (2ull * 0xD1B54A32D192ED03ull));
    uint64_t z = splitmix_mix(key + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull);
    double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    double a = bound[q];
    w[i] = (float)(-a + 2.0 * a * u);
}

int32_t model_xavier(ddg_model *m, uint64_t seed) {
    FlatOffsets fo = flat_offsets(m->d);
    const int d = m->d;
    std::vector<int> kind(fo.size, 0);
    std::vector<double> bound(fo.size, 0.0);
    auto mat = [&](int off, int fan_out, int fan_in) {
        double a = std::sqrt(6.0 / (fan_in + fan_out));
        for (int q = 0; q < fan_out * fan_in; ++q) { kind[off + q] = 1; bound[off + q] = a; }
    };
    for (int mm = 0; mm < 2; ++mm) {
        mat(fo.phi[mm][0], d, 2 * d + 3);
        mat(fo.phi[mm][2], d, d);
    }
    mat(fo.psi[0], d, 3 * d + 1);
    mat(fo.psi[2], d, d);
    mat(fo.dec[0], d, d);
    mat(fo.dec[2], 1, d);
    int *dk;
    double *db;
    DDG_CU(cudaMalloc(&dk, sizeof(int) * fo.size));
    DDG_CU(cudaMalloc(&db, sizeof(double) * fo.size));
    DDG_CU(cudaMemcpy(dk, kind.data(), sizeof(int) * fo.size, cudaMemcpyHostToDevice));
    DDG_CU(cudaMemcpy(db, bound.data(), sizeof(double) * fo.size, cudaMemcpyHostToDevice));
    long long n = (long long)m->kbar * fo.size;
    k_xavier<<<cdiv(n, 256), 256>>>(m->w, m->kbar, d, seed, dk, db, fo.size);
    DDG_LAUNCH_CHECK();
    DDG_CU(cudaDeviceSynchronize());
    cudaFree(dk);
    cudaFree(db);
    return DDG_OK;
}

// ---------------------------------------------------------------- the kernel
struct DssArgs {
    const float *weights;   // packed, kbar blocks
    int kbar;
    float alpha;
    const int *order;       // graph handed to CTA b
    const int *loc_ptr, *loc_nint, *nbr_ptr, *nbr_off, *sub_ptr, *sub_idx;
    const uint16_t *nbr;
    const float2 *loc_xy;
    const double *r;        // global residual (free nodes)
    const double *s;        // |R_i r| per subdomain
    double *corr;           // |R_i r| r~_i, sub_idx order
    int nmax, emax;         // shared-memory capacity in nodes and edges
    const int *stop;        // optional: skip all work when *stop != 0
    int *status;
    int test_skip_copy;     // failure test: never issue the first weight copy, so the bounded wait runs out
};

template <int P>
__global__ void __launch_bounds__(DSS_THREADS, 1) k_dss(DssArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    float *Wbuf = reinterpret_cast<float *>(smem + 128);
    float *Pb = Wbuf + 2 * BLOCK_FLOATS;                          // [nmax][20]
    float2 *xy = reinterpret_cast<float2 *>(Pb + (size_t)a.nmax * 2 * D);
    uint16_t *nptr = reinterpret_cast<uint16_t *>(xy + a.nmax);  // [nmax + 1]
    uint16_t *nbr = nptr + ((a.nmax + 1 + 7) & ~7);               // [emax]

    if (a.stop && *a.stop) return;
    const int tid = threadIdx.x;
    const int g = a.order[blockIdx.x];
    const int lp = a.loc_ptr[g];
    const int nl = a.loc_ptr[g + 1] - lp;
    const int k = a.loc_nint[g];
    const int *gptr = a.nbr_ptr + lp + g;
    const int ne = gptr[nl];
    const int s0 = a.sub_ptr[g];
    const double s = a.s[g];
    if (s == 0.0) {  // zero local residual: no correction
        for (int t = tid; t < k; t += DSS_THREADS) a.corr[s0 + t] = 0.0;
        return;
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0 && !a.test_skip_copy) bulk_load(Wbuf, a.weights, BLOCK_BYTES, &bar[0]);
    // stage the graph
    for (int q = tid; q < nl; q += DSS_THREADS) xy[q] = a.loc_xy[lp + q];
    for (int q = tid; q <= nl; q += DSS_THREADS) nptr[q] = (uint16_t)gptr[q];
    const uint16_t *gn = a.nbr + a.nbr_off[g];
    for (int e = tid; e < ne; e += DSS_THREADS) nbr[e] = gn[e];

    float h[P][D];
    float c[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        int j = p * DSS_THREADS + tid;
        c[p] = (j < k) ? (float)(a.r[a.sub_idx[s0 + j]] / s) : 0.f;
#pragma unroll
        for (int o = 0; o < D; ++o) h[p][o] = 0.f;
    }
    const float alpha = a.alpha;

    for (int blk = 0; blk < a.kbar; ++blk) {
        const int buf = blk & 1;
        const float *W = Wbuf + buf * BLOCK_FLOATS;
        const bool late = !mbar_wait(&bar[buf], (uint32_t)((blk >> 1) & 1));
        if (__syncthreads_or(late)) {
            // the weight copy did not arrive within about a second: report, give the copy one more
            // bounded wait (it must not land in shared memory this CTA no longer owns), and stop
            if (tid == 0) {
                raise_status(a.status, ST_TIMEOUT);
                if (!a.test_skip_copy || blk > 0) mbar_wait(&bar[buf], (uint32_t)((blk >> 1) & 1));
            }
            return;
        }
        if (tid == 0 && blk + 1 < a.kbar)
            bulk_load(Wbuf + (buf ^ 1) * BLOCK_FLOATS, a.weights + (size_t)(blk + 1) * BLOCK_FLOATS, BLOCK_BYTES,
                      &bar[buf ^ 1]);
        // phase A: neighbour-side projections of every node
#pragma unroll
        for (int p = 0; p < P; ++p) {
            int j = p * DSS_THREADS + tid;
            if (j < nl) {
                float po[D], pi[D];
#pragma unroll
                for (int o = 0; o < D; ++o) { po[o] = 0.f; pi[o] = 0.f; }
                mv_acc<D>(po, W + OFF_OUT + PHI_WB, h[p]);
                mv_acc<D>(pi, W + OFF_IN + PHI_WB, h[p]);
                float4 *dst = reinterpret_cast<float4 *>(Pb + (size_t)j * 2 * D);
                dst[0] = make_float4(po[0], po[1], po[2], po[3]);
                dst[1] = make_float4(po[4], po[5], po[6], po[7]);
                dst[2] = make_float4(po[8], po[9], pi[0], pi[1]);
                dst[3] = make_float4(pi[2], pi[3], pi[4], pi[5]);
                dst[4] = make_float4(pi[6], pi[7], pi[8], pi[9]);
            }
        }
        __syncthreads();
        // phase B: messages, aggregation, node update
#pragma unroll
        for (int p = 0; p < P; ++p) {
            int j = p * DSS_THREADS + tid;
            if (j < nl) {
                const bool inner = j < k;
                const float2 xj = xy[j];
                float Pa_o[D], Pa_i[D], So[D], Si[D];
                load_vec(Pa_o, W + OFF_OUT + PHI_B1);
                load_vec(Pa_i, W + OFF_IN + PHI_B1);
                mv_acc<D>(Pa_o, W + OFF_OUT + PHI_WA, h[p]);
                mv_acc<D>(Pa_i, W + OFF_IN + PHI_WA, h[p]);
#pragma unroll
                for (int o = 0; o < D; ++o) { So[o] = 0.f; Si[o] = 0.f; }
                int dout = 0, din = 0;
                const int e0 = nptr[j], e1 = nptr[j + 1];
                for (int e = e0; e < e1; ++e) {
                    const int l = nbr[e];
                    const float2 xl = xy[l];
                    const float dx = xl.x - xj.x, dy = xl.y - xj.y;
                    const float dn = sqrtf(dx * dx + dy * dy);
                    const float *pbl = Pb + (size_t)l * 2 * D;
                    if (l < k) {  // edge j -> l: out-message of j, feature d_jl = x_l - x_j
                        edge_msg(So, Pa_o, pbl, W + OFF_OUT + PHI_WE, dx, dy, dn);
                        ++dout;
                    }
                    if (inner) {  // edge l -> j: in-message of j, feature d_lj = x_j - x_l
                        edge_msg(Si, Pa_i, pbl + D, W + OFF_IN + PHI_WE, -dx, -dy, dn);
                        ++din;
                    }
                }
                float phi_o[D], phi_i[D];
                const float fo = (float)dout, fi = (float)din;
#pragma unroll
                for (int o = 0; o < D; ++o) {
                    phi_o[o] = fo * W[OFF_OUT + PHI_B2 + o];
                    phi_i[o] = fi * W[OFF_IN + PHI_B2 + o];
                }
                mv_acc<D>(phi_o, W + OFF_OUT + PHI_W2, So);
                mv_acc<D>(phi_i, W + OFF_IN + PHI_W2, Si);
                // Psi([h, c, phi_out, phi_in])
                float hid[D];
                load_vec(hid, W + OFF_PSI + PSI_B1);
                mv_acc<D>(hid, W + OFF_PSI + PSI_W1, h[p]);
                {
                    float cc[1] = {c[p]};
                    mv_acc<1>(hid, W + OFF_PSI + PSI_W1 + D * DP, cc);
                }
                mv_acc<D>(hid, W + OFF_PSI + PSI_W1 + (D + 1) * DP, phi_o);
                mv_acc<D>(hid, W + OFF_PSI + PSI_W1 + (2 * D + 1) * DP, phi_i);
#pragma unroll
                for (int o = 0; o < D; ++o) hid[o] = relu(hid[o]);
                float out[D];
                load_vec(out, W + OFF_PSI + PSI_B2);
                mv_acc<D>(out, W + OFF_PSI + PSI_W2, hid);
#pragma unroll
                for (int o = 0; o < D; ++o) h[p][o] = fmaf(alpha, out[o], h[p][o]);
            }
        }
        __syncthreads();
    }
    // decoder of the last block on the unknowns (Eq. 22)
    const float *W = Wbuf + ((a.kbar - 1) & 1) * BLOCK_FLOATS;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        int j = p * DSS_THREADS + tid;
        if (j < k) {
            float hid[D];
            load_vec(hid, W + OFF_DEC + DEC_B1);
            mv_acc<D>(hid, W + OFF_DEC + DEC_W1, h[p]);
            float y = W[OFF_DEC + DEC_B2];
#pragma unroll
            for (int o = 0; o < D; ++o) y = fmaf(W[OFF_DEC + DEC_W2 + o], relu(hid[o]), y);
            a.corr[s0 + j] = s * (double)y;
        }
    }
}

// ---------------------------------------------------------------- per-block schedule
// The same inference as k_dss, one launch per message-passing block: the
// block's weights travel as a kernel parameter, so every weight operand of the
// FMAs is read from the constant bank instead of shared memory, and shared
// memory holds only the neighbour projections.  Latents persist in global
// memory between launches (structure of arrays, h[o * n_total + node]); the
// graph (coordinates, adjacency) is read through the L1 cache.
struct __align__(16) BlockWeights {
    float w[BLOCK_FLOATS];
};

struct DssStepArgs {
    const int *order;
    const int *loc_ptr, *loc_nint, *nbr_ptr, *nbr_off, *sub_ptr, *sub_idx;
    const uint16_t *nbr;
    const float2 *loc_xy;
    const double *r, *s;
    double *corr;
    float *h;          // [D][n_total]
    float *c;          // [n_total]
    long long n_total;
    float alpha;
    int first, last;
    const int *stop;
};

template <int NIN, int OFF>
__device__ __forceinline__ void mvc_acc(float (&acc)[D], const BlockWeights &W, const float *x) {
#pragma unroll
    for (int i = 0; i < NIN; ++i) {
        const float xi = x[i];
#pragma unroll
        for (int o = 0; o < D; ++o) acc[o] = fmaf(W.w[OFF + i * DP + o], xi, acc[o]);
    }
}

template <int OFF>
__device__ __forceinline__ void loadc(float (&v)[D], const BlockWeights &W) {
#pragma unroll
    for (int o = 0; o < D; ++o) v[o] = W.w[OFF + o];
}

template <int OFF>
__device__ __forceinline__ void edge_msg_c(float (&S)[D], const float (&Pa)[D], const float *Pb, const BlockWeights &W,
                                           float ex, float ey, float en) {
#pragma unroll
    for (int o = 0; o < D; ++o) {
        float z = Pa[o] + Pb[o];
        z = fmaf(W.w[OFF + o], ex, z);
        z = fmaf(W.w[OFF + DP + o], ey, z);
        z = fmaf(W.w[OFF + 2 * DP + o], en, z);
        S[o] += relu(z);
    }
}

template <int P>
__global__ void __launch_bounds__(DSS_THREADS, 1) k_dss_step(const __grid_constant__ BlockWeights W,
                                                              const __grid_constant__ DssStepArgs a) {
    extern __shared__ __align__(16) float Pb[];  // [n_loc][2 D]
    if (a.stop && *a.stop) return;
    const int tid = threadIdx.x;
    const int g = a.order[blockIdx.x];
    const int lp = a.loc_ptr[g];
    const int nl = a.loc_ptr[g + 1] - lp;
    const int k = a.loc_nint[g];
    const int s0 = a.sub_ptr[g];
    const double s = a.s[g];
    if (s == 0.0) {
        if (a.last)
            for (int t = tid; t < k; t += DSS_THREADS) a.corr[s0 + t] = 0.0;
        return;
    }
    const int *gptr = a.nbr_ptr + lp + g;
    const uint16_t *gn = a.nbr + a.nbr_off[g];
    const float2 *xy = a.loc_xy + lp;
    float h[P][D];
    float c[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int j = p * DSS_THREADS + tid;
        if (j < nl) {
            if (a.first) {
                c[p] = (j < k) ? (float)(a.r[a.sub_idx[s0 + j]] / s) : 0.f;
                a.c[lp + j] = c[p];
#pragma unroll
                for (int o = 0; o < D; ++o) h[p][o] = 0.f;
            } else {
                c[p] = a.c[lp + j];
#pragma unroll
                for (int o = 0; o < D; ++o) h[p][o] = a.h[o * a.n_total + lp + j];
            }
        } else {
            c[p] = 0.f;
#pragma unroll
            for (int o = 0; o < D; ++o) h[p][o] = 0.f;
        }
    }
    // phase A
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int j = p * DSS_THREADS + tid;
        if (j < nl) {
            float po[D], pi[D];
#pragma unroll
            for (int o = 0; o < D; ++o) { po[o] = 0.f; pi[o] = 0.f; }
            mvc_acc<D, OFF_OUT + PHI_WB>(po, W, h[p]);
            mvc_acc<D, OFF_IN + PHI_WB>(pi, W, h[p]);
            float4 *dst = reinterpret_cast<float4 *>(Pb + (size_t)j * 2 * D);
            dst[0] = make_float4(po[0], po[1], po[2], po[3]);
            dst[1] = make_float4(po[4], po[5], po[6], po[7]);
            dst[2] = make_float4(po[8], po[9], pi[0], pi[1]);
            dst[3] = make_float4(pi[2], pi[3], pi[4], pi[5]);
            dst[4] = make_float4(pi[6], pi[7], pi[8], pi[9]);
        }
    }
    __syncthreads();
    // phase B
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int j = p * DSS_THREADS + tid;
        if (j < nl) {
            const bool inner = j < k;
            const float2 xj = xy[j];
            float Pa_o[D], Pa_i[D], So[D], Si[D];
            loadc<OFF_OUT + PHI_B1>(Pa_o, W);
            loadc<OFF_IN + PHI_B1>(Pa_i, W);
            mvc_acc<D, OFF_OUT + PHI_WA>(Pa_o, W, h[p]);
            mvc_acc<D, OFF_IN + PHI_WA>(Pa_i, W, h[p]);
#pragma unroll
            for (int o = 0; o < D; ++o) { So[o] = 0.f; Si[o] = 0.f; }
            int dout = 0, din = 0;
            const int e0 = gptr[j], e1 = gptr[j + 1];
            for (int e = e0; e < e1; ++e) {
                const int l = gn[e];
                const float2 xl = xy[l];
                const float dx = xl.x - xj.x, dy = xl.y - xj.y;
                const float dn = sqrtf(dx * dx + dy * dy);
                const float *pbl = Pb + (size_t)l * 2 * D;
                if (l < k) {
                    edge_msg_c<OFF_OUT + PHI_WE>(So, Pa_o, pbl, W, dx, dy, dn);
                    ++dout;
                }
                if (inner) {
                    edge_msg_c<OFF_IN + PHI_WE>(Si, Pa_i, pbl + D, W, -dx, -dy, dn);
                    ++din;
                }
            }
            float phi_o[D], phi_i[D];
            const float fo = (float)dout, fi = (float)din;
#pragma unroll
            for (int o = 0; o < D; ++o) {
                phi_o[o] = fo * W.w[OFF_OUT + PHI_B2 + o];
                phi_i[o] = fi * W.w[OFF_IN + PHI_B2 + o];
            }
            mvc_acc<D, OFF_OUT + PHI_W2>(phi_o, W, So);
            mvc_acc<D, OFF_IN + PHI_W2>(phi_i, W, Si);
            float hid[D];
            loadc<OFF_PSI + PSI_B1>(hid, W);
            mvc_acc<D, OFF_PSI + PSI_W1>(hid, W, h[p]);
            {
                float cc[1] = {c[p]};
                mvc_acc<1, OFF_PSI + PSI_W1 + D * DP>(hid, W, cc);
            }
            mvc_acc<D, OFF_PSI + PSI_W1 + (D + 1) * DP>(hid, W, phi_o);
            mvc_acc<D, OFF_PSI + PSI_W1 + (2 * D + 1) * DP>(hid, W, phi_i);
#pragma unroll
            for (int o = 0; o < D; ++o) hid[o] = relu(hid[o]);
            float out[D];
            loadc<OFF_PSI + PSI_B2>(out, W);
            mvc_acc<D, OFF_PSI + PSI_W2>(out, W, hid);
#pragma unroll
            for (int o = 0; o < D; ++o) h[p][o] = fmaf(a.alpha, out[o], h[p][o]);
            if (a.last) {
                if (inner) {
                    float dh[D];
                    loadc<OFF_DEC + DEC_B1>(dh, W);
                    mvc_acc<D, OFF_DEC + DEC_W1>(dh, W, h[p]);
                    float y = W.w[OFF_DEC + DEC_B2];
#pragma unroll
                    for (int o = 0; o < D; ++o) y = fmaf(W.w[OFF_DEC + DEC_W2 + o], relu(dh[o]), y);
                    a.corr[s0 + j] = s * (double)y;
                }
            } else {
#pragma unroll
                for (int o = 0; o < D; ++o) a.h[o * a.n_total + lp + j] = h[p][o];
            }
        }
    }
}

// ---------------------------------------------------------------- chunked per-block schedule
// Each graph is cut into chunks of at most 2 * T consecutive local nodes; a CTA
// of T threads owns one chunk.  Its shared memory holds the neighbour
// projections of the chunk's nodes and of their neighbours only, addressed by
// chunk-local ids built at set-up, so several CTAs share an SM and every SM
// receives work even when there are fewer graphs than SMs.  Latents alternate
// between two global buffers, because a chunk reads the latents of nodes that
// other chunks update in the same launch.

template <int T>
__global__ void __launch_bounds__(T, 65536 / (T * 112)) k_dss_chunk(const __grid_constant__ BlockWeights W,
                                                 const __grid_constant__ ChunkArgs a) {
    extern __shared__ __align__(16) float Pb[];  // [needed][2 D]
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
    if (s == 0.0) {
        if (a.last)
            for (int t = tid; t < own; t += T)
                if (n0 + t < k) a.corr[s0 + n0 + t] = 0.0;
        return;
    }
    // phase A: projections of every needed node
    for (int u = tid; u < nn; u += T) {
        const int j = need[u];
        float h[D], po[D], pi[D];
        if (a.first) {
#pragma unroll
            for (int o = 0; o < D; ++o) h[o] = 0.f;
        } else {
#pragma unroll
            for (int o = 0; o < D; ++o) h[o] = a.h_in[o * a.n_total + lp + j];
        }
#pragma unroll
        for (int o = 0; o < D; ++o) { po[o] = 0.f; pi[o] = 0.f; }
        mvc_acc<D, OFF_OUT + PHI_WB>(po, W, h);
        mvc_acc<D, OFF_IN + PHI_WB>(pi, W, h);
        float4 *dst = reinterpret_cast<float4 *>(Pb + (size_t)u * 2 * D);
        dst[0] = make_float4(po[0], po[1], po[2], po[3]);
        dst[1] = make_float4(po[4], po[5], po[6], po[7]);
        dst[2] = make_float4(po[8], po[9], pi[0], pi[1]);
        dst[3] = make_float4(pi[2], pi[3], pi[4], pi[5]);
        dst[4] = make_float4(pi[6], pi[7], pi[8], pi[9]);
    }
    __syncthreads();
    const int *aptr = a.adj_ptr + a.c_adj_off[q];
    const uint16_t *adj = a.adj + a.c_adj_base[q];
    const float2 *xy = a.loc_xy + lp;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int u = p * T + tid;  // chunk-local id of an own node
        if (u >= own) continue;
        const int j = n0 + u;       // graph-local id
        const bool inner = j < k;
        float h[D], c;
        if (a.first) {
            c = inner ? (float)(a.r[a.sub_idx[s0 + j]] / s) : 0.f;
            a.c[lp + j] = c;
#pragma unroll
            for (int o = 0; o < D; ++o) h[o] = 0.f;
        } else {
            c = a.c[lp + j];
#pragma unroll
            for (int o = 0; o < D; ++o) h[o] = a.h_in[o * a.n_total + lp + j];
        }
        const float2 xj = xy[j];
        float Pa_o[D], Pa_i[D], So[D], Si[D];
        loadc<OFF_OUT + PHI_B1>(Pa_o, W);
        loadc<OFF_IN + PHI_B1>(Pa_i, W);
        mvc_acc<D, OFF_OUT + PHI_WA>(Pa_o, W, h);
        mvc_acc<D, OFF_IN + PHI_WA>(Pa_i, W, h);
#pragma unroll
        for (int o = 0; o < D; ++o) { So[o] = 0.f; Si[o] = 0.f; }
        int dout = 0, din = 0;
        for (int e = aptr[u]; e < aptr[u + 1]; ++e) {
            const int v = adj[e];          // chunk-local
            const int l = need[v];         // graph-local
            const float2 xl = xy[l];
            const float dx = xl.x - xj.x, dy = xl.y - xj.y;
            const float dn = sqrtf(dx * dx + dy * dy);
            const float *pbl = Pb + (size_t)v * 2 * D;
            if (l < k) {
                edge_msg_c<OFF_OUT + PHI_WE>(So, Pa_o, pbl, W, dx, dy, dn);
                ++dout;
            }
            if (inner) {
                edge_msg_c<OFF_IN + PHI_WE>(Si, Pa_i, pbl + D, W, -dx, -dy, dn);
                ++din;
            }
        }
        float phi_o[D], phi_i[D];
        const float fo = (float)dout, fi = (float)din;
#pragma unroll
        for (int o = 0; o < D; ++o) {
            phi_o[o] = fo * W.w[OFF_OUT + PHI_B2 + o];
            phi_i[o] = fi * W.w[OFF_IN + PHI_B2 + o];
        }
        mvc_acc<D, OFF_OUT + PHI_W2>(phi_o, W, So);
        mvc_acc<D, OFF_IN + PHI_W2>(phi_i, W, Si);
        float hid[D];
        loadc<OFF_PSI + PSI_B1>(hid, W);
        mvc_acc<D, OFF_PSI + PSI_W1>(hid, W, h);
        {
            float cc[1] = {c};
            mvc_acc<1, OFF_PSI + PSI_W1 + D * DP>(hid, W, cc);
        }
        mvc_acc<D, OFF_PSI + PSI_W1 + (D + 1) * DP>(hid, W, phi_o);
        mvc_acc<D, OFF_PSI + PSI_W1 + (2 * D + 1) * DP>(hid, W, phi_i);
#pragma unroll
        for (int o = 0; o < D; ++o) hid[o] = relu(hid[o]);
        float out[D];
        loadc<OFF_PSI + PSI_B2>(out, W);
        mvc_acc<D, OFF_PSI + PSI_W2>(out, W, hid);
#pragma unroll
        for (int o = 0; o < D; ++o) h[o] = fmaf(a.alpha, out[o], h[o]);
        if (a.last) {
            if (inner) {
                float dh[D];
                loadc<OFF_DEC + DEC_B1>(dh, W);
                mvc_acc<D, OFF_DEC + DEC_W1>(dh, W, h);
                float y = W.w[OFF_DEC + DEC_B2];
#pragma unroll
                for (int o = 0; o < D; ++o) y = fmaf(W.w[OFF_DEC + DEC_W2 + o], relu(dh[o]), y);
                a.corr[s0 + j] = s * (double)y;
            }
        } else {
#pragma unroll
            for (int o = 0; o < D; ++o) a.h_out[o * a.n_total + lp + j] = h[o];
        }
    }
}

// ---------------------------------------------------------------- fused global-chunk schedule
// Schedule 3.  Chunks are equal ranges of the concatenated graphs' nodes (a chunk
// may hold the end of one graph and the start of the next), as many as fill the
// SMs' resident CTAs a whole number of times, so every SM gets the same work in
// every block.  Own nodes are processed in decreasing order of their messages,
// so the lanes of a warp run edge loops of equal length.  Weights come in the
// composed layout (dss_layout.cuh) and the arithmetic runs on packed pairs of
// FP32 lanes: a matrix-vector product issues one fma.rn.f32x2 per two outputs.
// Out-messages to halo neighbours are masked (multiplied by 0) rather than
// branched over.  Shared memory: per needed node its neighbour projections as
// five float4 (Wb_out h pair m, Wb_in h pair m) and its scaled coordinates.
template <int T>
__device__ __forceinline__ void fused_project(const FusedWeights &W, const float (&h)[D], float2 xy, float4 *dst) {
    const f2_t *Wp = reinterpret_cast<const f2_t *>(W.w);
    f2_t acc[D];
    {
        const f2_t x2 = f2_pack(xy.x, xy.x), y2 = f2_pack(xy.y, xy.y);
#pragma unroll
        for (int q = 0; q < D; ++q)
            acc[q] = f2_fma(Wp[(F_XB + 2 * D) / 2 + q], y2, f2_fma(Wp[F_XB / 2 + q], x2, 0ull));
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const f2_t xi = f2_pack(h[i], h[i]);
#pragma unroll
        for (int q = 0; q < D; ++q) acc[q] = f2_fma(Wp[(F_HB + i * 2 * D) / 2 + q], xi, acc[q]);
    }
#pragma unroll
    for (int m = 0; m < D / 2; ++m) {
        float a0, a1, b0, b1;
        f2_unpack(acc[2 * m], a0, a1);
        f2_unpack(acc[2 * m + 1], b0, b1);
        dst[m] = make_float4(a0, a1, b0, b1);
    }
}

// shared memory of one chunk: per needed node its neighbour projections (five float4) and
// scaled coordinates (float2); per own node its latent row (three float4, copied from the
// loads of the projection phase for phase B)
__host__ __device__ __forceinline__ size_t fused_smem(int nn, int own) {
    return (size_t)nn * 5 * sizeof(float4) + (size_t)own * 3 * sizeof(float4) + (size_t)nn * sizeof(float2);
}

// One CTA of schedule 3 on chunk q of the plan in `a`; first/last mark the first and last
// message-passing block, h_in/h_out the latent rows read and written.
template <int T>
__device__ __forceinline__ void fused_chunk(const FusedWeights &W, const ChunkArgs &a, int q, bool first, bool last,
                                            const float *h_in, float *h_out) {
    extern __shared__ __align__(16) float4 smem4[];
    if (a.stop && *a.stop) return;
    const int tid = threadIdx.x;
    const int own = a.c_own[q];
    const int nn = a.c_need_n[q];
    const int *need = a.need + a.c_need_off[q];  // local-node ids over all graphs: own nodes first
    const int *APTR = a.adj_ptr + a.c_adj_off[q];      // [own + 1]
    const uint2 *ADJX = a.adjx + a.c_adj_base[q];      // {chunk-local id, |d|}, each node's unknowns first
    const int4 *INFO = a.info + a.c_n0[q];             // [own] {node, corr idx, r idx, graph | dout << 24}
    float4 *Pb = smem4;                                               // [nn][5]
    float4 *HS = Pb + (size_t)nn * 5;                                 // [own][3] latent rows of own nodes
    float2 *XY = reinterpret_cast<float2 *>(HS + (size_t)own * 3);    // [nn]
    const f2_t *Wp = reinterpret_cast<const f2_t *>(W.w);
    const float4 *hrow_in = reinterpret_cast<const float4 *>(h_in);  // rows of 12: h[10], c, 0
    // the plan data of this thread's own nodes and of phase A's first needed node: set-up data,
    // loaded before waiting for the previous block
    int4 pinf[2];
    int pe0[2], pe1[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int u = p * T + tid;
        pinf[p] = make_int4(0, -1, 0, 0);
        pe0[p] = pe1[p] = 0;
        if (u < own) {
            pinf[p] = INFO[u];
            pe0[p] = APTR[u];
            pe1[p] = APTR[u + 1];
        }
    }
    const int node0 = tid < nn ? need[tid] : 0;
    const float2 xy0 = tid < nn ? a.loc_xy[node0] : make_float2(0.f, 0.f);
    // launched as a programmatic dependent of the previous block: everything above reads
    // set-up data only; wait here until the previous launch's latents are complete and visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // phase A: projections and coordinates of every needed node
    // software-pipelined: the next node's latent row and coordinates are loaded while this one is
    // projected (phase A holds far fewer live values than phase B, so this costs no occupancy)
    {
        float h[D], cl = 0.f;
        float2 xy = make_float2(0.f, 0.f);
#pragma unroll
        for (int o = 0; o < D; ++o) h[o] = 0.f;
        if (tid < nn) {
            xy = xy0;
            if (!first) load_hrow(hrow_in, node0, h, cl);
        }
        for (int u = tid; u < nn; u += T) {
            float hn[D], cn = 0.f;
            float2 xyn = make_float2(0.f, 0.f);
#pragma unroll
            for (int o = 0; o < D; ++o) hn[o] = 0.f;
            if (u + T < nn) {
                const int nnode = need[u + T];
                xyn = a.loc_xy[nnode];
                if (!first) load_hrow(hrow_in, nnode, hn, cn);
            }
            fused_project<T>(W, h, xy, Pb + (size_t)u * 5);  // (h = 0 in the first block)
            XY[u] = xy;
            if (u < own) {  // own nodes keep their row for phase B
                HS[3 * (size_t)u] = make_float4(h[0], h[1], h[2], h[3]);
                HS[3 * (size_t)u + 1] = make_float4(h[4], h[5], h[6], h[7]);
                HS[3 * (size_t)u + 2] = make_float4(h[8], h[9], cl, 0.f);
            }
#pragma unroll
            for (int o = 0; o < D; ++o) h[o] = hn[o];
            cl = cn;
            xy = xyn;
        }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int u = p * T + tid;
        if (u >= own) continue;
        const int4 inf = pinf[p];
        const int node = inf.x;
        const bool inner = inf.y >= 0;
        float hp[D], c;  // from the copy phase A left in shared memory
        if (first) {
#pragma unroll
            for (int o = 0; o < D; ++o) hp[o] = 0.f;
            const double s = a.s[inf.w & 0xffffff];
            c = (inner && s != 0.0) ? (float)(a.r[inf.z] / s) : 0.f;
        } else {
            load_hrow(HS, u, hp, c);
        }
        const float2 xj = XY[u];
        const int e0 = pe0[p], e1 = pe1[p];
        f2_t so[D / 2], si[D / 2], pao[D / 2], pai[D / 2];
        const int n_out = min((int)((unsigned)inf.w >> 24), e1 - e0);  // out-messages (neighbours that are unknowns)
        const float dout = (float)n_out;
#pragma unroll
        for (int m = 0; m < D / 2; ++m) {
            so[m] = 0ull;
            si[m] = 0ull;
            pao[m] = Wp[F_BA / 2 + m];
            pai[m] = Wp[(F_BA + D) / 2 + m];
        }
        f2_mv<F_HA, 3 * D>(pao, Wp, hp);
        if (inner) f2_mv<F_HA + D, 3 * D>(pai, Wp, hp);
        {
            const f2_t x2 = f2_pack(xj.x, xj.x), y2 = f2_pack(xj.y, xj.y);
#pragma unroll
            for (int m = 0; m < D / 2; ++m) {
                pao[m] = f2_fma(Wp[(F_NXA + 2 * D) / 2 + m], y2, f2_fma(Wp[F_NXA / 2 + m], x2, pao[m]));
                pai[m] = f2_fma(Wp[(F_NXA + 3 * D) / 2 + m], y2, f2_fma(Wp[(F_NXA + D) / 2 + m], x2, pai[m]));
            }
        }
        // messages: with q = pb + We_|d| |d|, relu(pa + q) = max(q, -pa) + pa, so the loops sum
        // max(q, -pa) and (messages) * pa is added after them; each node lists its unknown
        // neighbours (out- and in-messages) before its halo neighbours (in-messages only), with the
        // edge length precomputed; the next entry is loaded one iteration ahead
        {
            const uint2 *ap = ADJX + e0, *const ae = ADJX + e1, *const au = ADJX + e0 + n_out;
            uint2 nxt = ap < ae ? *ap : make_uint2(0u, 0u);
            for (; ap < au; ++ap) {
                const uint2 ent = nxt;
                if (ap + 1 < ae) nxt = ap[1];
                const float dn = __uint_as_float(ent.y);
                const f2_t dn2 = f2_pack(dn, dn);
                const float4 *pb = Pb + (size_t)ent.x * 5;
#pragma unroll
                for (int m = 0; m < D / 2; ++m) {  // one 16-byte shared load per output pair of both messages
                    const float4 t = pb[m];
                    so[m] = f2_add(so[m], f2_max_neg(f2_fma(Wp[(F_WEO + 2 * D) / 2 + m], dn2, f2_pack(t.x, t.y)), pao[m]));
                    if (inner)
                        si[m] = f2_add(si[m],
                                       f2_max_neg(f2_fma(Wp[(F_WEI + 2 * D) / 2 + m], dn2, f2_pack(t.z, t.w)), pai[m]));
                }
            }
            if (inner) {
                for (; ap < ae; ++ap) {
                    const uint2 ent = nxt;
                    if (ap + 1 < ae) nxt = ap[1];
                    const float dn = __uint_as_float(ent.y);
                    const f2_t dn2 = f2_pack(dn, dn);
                    const float4 *pb = Pb + (size_t)ent.x * 5;
#pragma unroll
                    for (int m = 0; m < D / 2; ++m) {
                        const float4 t = pb[m];
                        si[m] = f2_add(si[m],
                                       f2_max_neg(f2_fma(Wp[(F_WEI + 2 * D) / 2 + m], dn2, f2_pack(t.z, t.w)), pai[m]));
                    }
                }
            }
            const float fi = inner ? (float)(e1 - e0) : 0.f;
            const f2_t fo2 = f2_pack(dout, dout), fi2 = f2_pack(fi, fi);
#pragma unroll
            for (int m = 0; m < D / 2; ++m) {
                so[m] = f2_fma(fo2, pao[m], so[m]);
                si[m] = f2_fma(fi2, pai[m], si[m]);
            }
        }
        const float din = inner ? (float)(e1 - e0) : 0.f;
        // Psi hidden layer on [h, c, phi_out, phi_in] with the second message layers composed in
        f2_t hid[D / 2];
#pragma unroll
        for (int m = 0; m < D / 2; ++m) hid[m] = Wp[(F_BA + 2 * D) / 2 + m];
        f2_mv<F_HA + 2 * D, 3 * D>(hid, Wp, hp);
        {
            const f2_t cc = f2_pack(c, c), dd = f2_pack(dout, dout), di = f2_pack(din, din);
#pragma unroll
            for (int m = 0; m < D / 2; ++m) {
                hid[m] = f2_fma(Wp[F_VC / 2 + m], cc, hid[m]);
                hid[m] = f2_fma(Wp[F_VO / 2 + m], dd, hid[m]);
                hid[m] = f2_fma(Wp[F_VI / 2 + m], di, hid[m]);
            }
        }
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
        // h += alpha (Psi_W2 relu(hid) + Psi_b2)
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
            const f2_t hv = f2_add(f2_pack(hp[2 * m], hp[2 * m + 1]), out[m]);
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
            float4 *hrow_out = reinterpret_cast<float4 *>(h_out) + 3 * (size_t)node;
            hrow_out[0] = make_float4(hn[0], hn[1], hn[2], hn[3]);
            hrow_out[1] = make_float4(hn[4], hn[5], hn[6], hn[7]);
            hrow_out[2] = make_float4(hn[8], hn[9], c, 0.f);
        }
    }
    // this CTA's writes are issued: the next block's CTAs may be scheduled (they still wait
    // for the whole grid at their griddepcontrol.wait)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <int T>
__global__ void __launch_bounds__(T, 65536 / (T * 128))
    k_dss_fused(const __grid_constant__ FusedWeights W, const __grid_constant__ ChunkArgs a) {
    fused_chunk<T>(W, a, blockIdx.x, a.first, a.last, a.h_in, a.h_out);
}

// Several problems' graphs in one launch (the request loop's fused GNN step): CTA b runs
// chunk b - cpre[i] of problem i, where cpre[i] <= b < cpre[i + 1].  Every problem's
// descriptor holds its latent buffers in block-0 orientation; odd blocks swap them.
constexpr int MAX_GROUP = 32;
struct GroupArgs {
    int n;                      // problems in the group
    int first, last, odd;       // block flags
    int cpre[MAX_GROUP + 1];    // chunk prefix sums
    const ChunkArgs *args;      // [n] descriptors (device)
};

template <int T>
__global__ void __launch_bounds__(T, 65536 / (T * 128))
    k_dss_fused_group(const __grid_constant__ FusedWeights W, const __grid_constant__ GroupArgs g) {
    int lo = 0, hi = g.n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (g.cpre[mid] <= (int)blockIdx.x) lo = mid; else hi = mid;
    }
    const ChunkArgs &a = g.args[lo];
    fused_chunk<T>(W, a, blockIdx.x - g.cpre[lo], g.first != 0, g.last != 0, g.odd ? a.h_out : a.h_in,
                   g.odd ? const_cast<float *>(a.h_in) : a.h_out);
}

// Set-up of a global chunk plan, one CTA per chunk: the chunk's own nodes are the
// local-node range [c_n0, c_n0 + c_own) of the concatenated graphs (a chunk may
// span two graphs; edges never do).  Pass 0 counts needed nodes and adjacency
// entries; pass 1 lists the own nodes in decreasing order of their messages per
// block, then the outside neighbours (ascending), and writes the chunk-local
// adjacency with bit 15 set for neighbours that are unknowns.
__global__ void __launch_bounds__(256) k_gchunk_build(const int *c_n0, const int *c_own, const int *gid,
                                                      const int *loc_ptr, const int *loc_nint, const int *nbr_ptr,
                                                      const int *nbr_off, const uint16_t *nbr, const int *sub_ptr,
                                                      const int *sub_idx, int pass, int *need_n, int *adj_n,
                                                      const int *need_off, int *need, const int *adj_off,
                                                      int *adj_ptr, const int *adj_base, uint16_t *adj, int4 *info,
                                                      const float2 *loc_xy, uint2 *adjx, int *st) {
    constexpr int NT = 256, MAXN = 2048, MAXO = 512;
    __shared__ int cand[MAXN];
    __shared__ int work[MAXO], slot[MAXO], order[MAXO], sptr[MAXO + 1];
    __shared__ int cnt, uniq;
    const int q = blockIdx.x;
    const int o0 = c_n0[q], own = c_own[q];
    if (own > MAXO) {
        if (threadIdx.x == 0) raise_status(st, ST_TOO_LARGE);
        return;
    }
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    // neighbours of own node t: local ids of its graph, as global local-node ids
    auto row = [&](int t, int &g, int &lp, int &e0, int &e1) {
        const int u = o0 + t;
        g = gid[u];
        lp = loc_ptr[g];
        const int *gptr = nbr_ptr + lp + g;
        e0 = gptr[u - lp];
        e1 = gptr[u - lp + 1];
    };
    for (int t = threadIdx.x; t < own; t += NT) {
        int g, lp, e0, e1;
        row(t, g, lp, e0, e1);
        const uint16_t *gn = nbr + nbr_off[g];
        for (int e = e0; e < e1; ++e) {
            const int l = lp + gn[e];
            if (l < o0 || l >= o0 + own) {
                const int pos = atomicAdd(&cnt, 1);
                if (pos < MAXN) cand[pos] = l;
            }
        }
    }
    __syncthreads();
    const int m = cnt;
    if (m > MAXN) {
        if (threadIdx.x == 0) raise_status(st, ST_TOO_LARGE);
        return;
    }
    int N = 1;
    while (N < m) N <<= 1;
    for (int t = m + threadIdx.x; t < N; t += NT) cand[t] = INT_MAX;
    __syncthreads();
    for (int kk = 2; kk <= N; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int t = threadIdx.x; t < N; t += NT) {
                const int r = t ^ jj;
                if (r > t) {
                    const bool up = (t & kk) == 0;
                    const int x = cand[t], y = cand[r];
                    if ((x > y) == up) {
                        cand[t] = y;
                        cand[r] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        int u = 0;
        for (int t = 0; t < m; ++t)
            if (t == 0 || cand[t] != cand[t - 1]) cand[u++] = cand[t];
        uniq = u;
    }
    __syncthreads();
    const int ext = uniq;
    if (pass == 0) {
        if (threadIdx.x == 0) {
            need_n[q] = own + ext;
            int tot = 0;
            for (int t = 0; t < own; ++t) {
                int g, lp, e0, e1;
                row(t, g, lp, e0, e1);
                tot += e1 - e0;
            }
            adj_n[q] = tot;
        }
        return;
    }
    for (int t = threadIdx.x; t < own; t += NT) {
        int g, lp, e0, e1;
        row(t, g, lp, e0, e1);
        const uint16_t *gn = nbr + nbr_off[g];
        const int k = loc_nint[g];
        int w = 0;
        for (int e = e0; e < e1; ++e) w += gn[e] < k ? 1 : 0;
        if (o0 + t - lp < k) w += e1 - e0;
        work[t] = w;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < own; t += NT) {  // rank: more messages first, then lower id
        int r = 0;
        for (int u = 0; u < own; ++u) r += (work[u] > work[t] || (work[u] == work[t] && u < t)) ? 1 : 0;
        slot[t] = r;
        order[r] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sptr[0] = 0;
        for (int r = 0; r < own; ++r) {
            int g, lp, e0, e1;
            row(order[r], g, lp, e0, e1);
            sptr[r + 1] = sptr[r] + e1 - e0;
        }
    }
    __syncthreads();
    int *nd = need + need_off[q];
    int *ap = adj_ptr + adj_off[q];
    uint16_t *ad = adj + adj_base[q];
    for (int r = threadIdx.x; r < own; r += NT) {
        const int u = o0 + order[r];
        const int g = gid[u];
        const int j = u - loc_ptr[g];
        const bool in = j < loc_nint[g];
        nd[r] = u;
        int dout = 0;  // out-messages per block: neighbours that are unknowns
        {
            const int *gptr = nbr_ptr + loc_ptr[g] + g;
            const uint16_t *gn = nbr + nbr_off[g];
            for (int e = gptr[j]; e < gptr[j + 1]; ++e) dout += gn[e] < loc_nint[g] ? 1 : 0;
        }
        info[o0 + r] = make_int4(u, in ? sub_ptr[g] + j : -1, in ? sub_idx[sub_ptr[g] + j] : -1,
                                 g | (min(dout, 255) << 24));
    }
    for (int t = threadIdx.x; t < ext; t += NT) nd[own + t] = cand[t];
    for (int r = threadIdx.x; r <= own; r += NT) ap[r] = sptr[r];
    // schedule 4 (adjx given): each node's unknown neighbours first, with the edge length
    for (int r = threadIdx.x; r < own; r += NT) {
        int g, lp, e0, e1;
        row(order[r], g, lp, e0, e1);
        const uint16_t *gn = nbr + nbr_off[g];
        const int k = loc_nint[g];
        const float2 xj = loc_xy[o0 + order[r]];
        int pos = sptr[r];
        for (int pass2 = 0; pass2 < (adjx ? 2 : 1); ++pass2) {
            for (int e = e0; e < e1; ++e) {
                const bool unknown = gn[e] < k;
                if (adjx && unknown != (pass2 == 0)) continue;
                const int l = lp + gn[e];
                int v;
                if (l >= o0 && l < o0 + own) {
                    v = slot[l - o0];
                } else {
                    int lo = 0, hi = ext;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (cand[mid] < l) lo = mid + 1; else hi = mid;
                    }
                    v = own + lo;
                }
                ad[pos] = (uint16_t)(v | (unknown ? 0x8000 : 0));
                if (adjx) {
                    const float2 xl = loc_xy[l];
                    const float dx = xl.x - xj.x, dy = xl.y - xj.y;
                    adjx[adj_base[q] + pos] = make_uint2((unsigned)v, __float_as_uint(sqrtf(fmaf(dx, dx, dy * dy))));
                }
                ++pos;
            }
        }
    }
}

// set-up of the chunks of one graph per CTA: needed-node lists and chunk-local adjacency.
// Pass 0 counts (needed nodes, adjacency entries) per chunk; pass 1 fills.
constexpr int CH_T = 256;
constexpr int CH_MAX_NEED = 2048;

__global__ void __launch_bounds__(CH_T) k_chunk_build(const int *c_graph, const int *c_n0, const int *c_own,
                                                      const int *loc_ptr, const int *nbr_ptr, const int *nbr_off,
                                                      const uint16_t *nbr, int pass, int *need_n, int *adj_n,
                                                      const int *need_off, int *need, const int *adj_off,
                                                      int *adj_ptr, const int *adj_base, uint16_t *adj, int *st) {
    __shared__ int cand[CH_MAX_NEED];
    __shared__ int cnt;
    const int q = blockIdx.x;
    const int g = c_graph[q], n0 = c_n0[q], own = c_own[q];
    const int lp = loc_ptr[g];
    const int *gptr = nbr_ptr + lp + g;
    const uint16_t *gn = nbr + nbr_off[g];
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < own; t += CH_T) {
        const int j = n0 + t;
        for (int e = gptr[j]; e < gptr[j + 1]; ++e) {
            const int l = gn[e];
            if (l < n0 || l >= n0 + own) {
                int pos = atomicAdd(&cnt, 1);
                if (pos < CH_MAX_NEED) cand[pos] = l;
            }
        }
    }
    __syncthreads();
    const int m = cnt;
    if (m > CH_MAX_NEED) {
        if (threadIdx.x == 0) raise_status(st, ST_TOO_LARGE);
        return;
    }
    int N = 1;
    while (N < m) N <<= 1;
    for (int t = m + threadIdx.x; t < N; t += CH_T) cand[t] = INT_MAX;
    __syncthreads();
    for (int kk = 2; kk <= N; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < N; t += CH_T) {
                int r = t ^ j;
                if (r > t) {
                    bool up = (t & kk) == 0;
                    int x = cand[t], y = cand[r];
                    if ((x > y) == up) { cand[t] = y; cand[r] = x; }
                }
            }
            __syncthreads();
        }
    }
    __shared__ int uniq;
    if (threadIdx.x == 0) {
        int u = 0;
        for (int t = 0; t < m; ++t)
            if (t == 0 || cand[t] != cand[t - 1]) cand[u++] = cand[t];
        uniq = u;
    }
    __syncthreads();
    const int ext = uniq;
    if (pass == 0) {
        if (threadIdx.x == 0) {
            need_n[q] = own + ext;
            adj_n[q] = gptr[n0 + own] - gptr[n0];
        }
        return;
    }
    int *nd = need + need_off[q];
    for (int t = threadIdx.x; t < own; t += CH_T) nd[t] = n0 + t;
    for (int t = threadIdx.x; t < ext; t += CH_T) nd[own + t] = cand[t];
    int *ap = adj_ptr + adj_off[q];
    uint16_t *ad = adj + adj_base[q];
    const int e00 = gptr[n0];
    for (int t = threadIdx.x; t <= own; t += CH_T) ap[t] = gptr[n0 + t] - e00;
    for (int t = threadIdx.x; t < own; t += CH_T) {
        const int j = n0 + t;
        for (int e = gptr[j]; e < gptr[j + 1]; ++e) {
            const int l = gn[e];
            int v;
            if (l >= n0 && l < n0 + own) {
                v = l - n0;
            } else {
                int lo = 0, hi = ext;
                while (lo < hi) {
                    int mid = (lo + hi) >> 1;
                    if (cand[mid] < l) lo = mid + 1; else hi = mid;
                }
                v = own + lo;
            }
            ad[e - e00] = (uint16_t)v;
        }
    }
}

void chunk_free(ddg_problem *p) {
    dfree_all(p->ctx, p->chunk.allocs);  // keeps the stage's stream settings
    ChunkPlan empty;
    p->chunk.T = p->chunk.nchunks = p->chunk.max_need = 0;
    p->chunk.c_graph = p->chunk.c_n0 = p->chunk.c_own = p->chunk.c_need_off = p->chunk.c_need_n = nullptr;
    p->chunk.need = p->chunk.c_adj_off = p->chunk.adj_ptr = p->chunk.c_adj_base = nullptr;
    p->chunk.adj = nullptr;
    p->chunk.adjx = nullptr;
    p->chunk.gid = nullptr;
    p->chunk.info = nullptr;
    p->chunk.global = false;
    p->chunk.tc = false;
    (void)empty;
}

int32_t chunk_build(ddg_problem *p, int T) {
    ddg_ctx *c = p->ctx;
    cudaStream_t s = p->stream;
    chunk_free(p);
    ChunkPlan &cp = p->chunk;
    const int K = p->K;
    std::vector<int> lp(K + 1);
    DDG_CU(cudaMemcpyAsync(lp.data(), p->loc_ptr, sizeof(int) * (K + 1), cudaMemcpyDeviceToHost, s));
    DDG_CU(cudaStreamSynchronize(s));
    std::vector<int> cg, cn0, cown;
    for (int g = 0; g < K; ++g) {
        const int nl = lp[g + 1] - lp[g];
        const int nq = std::max(1, cdiv(nl, 2 * T));
        const int cs = cdiv(nl, nq);
        for (int q = 0; q < nq; ++q) {
            cg.push_back(g);
            cn0.push_back(q * cs);
            cown.push_back(std::min(cs, nl - q * cs));
        }
    }
    const int nc = (int)cg.size();
    cp.T = T;
    cp.nchunks = nc;
    DDG_TRY(dalloc(c, cp.allocs, &cp.c_graph, nc));
    DDG_TRY(dalloc(c, cp.allocs, &cp.c_n0, nc));
    DDG_TRY(dalloc(c, cp.allocs, &cp.c_own, nc));
    DDG_TRY(dalloc(c, cp.allocs, &cp.c_need_off, nc));
    DDG_TRY(dalloc(c, cp.allocs, &cp.c_need_n, nc));
    DDG_TRY(dalloc(c, cp.allocs, &cp.c_adj_off, nc));
    DDG_TRY(dalloc(c, cp.allocs, &cp.c_adj_base, nc));
    DDG_CU(cudaMemcpyAsync(cp.c_graph, cg.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    DDG_CU(cudaMemcpyAsync(cp.c_n0, cn0.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    DDG_CU(cudaMemcpyAsync(cp.c_own, cown.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    Scratch sc(s);
    int *adj_n = nullptr;
    DDG_CU(sc.get(&adj_n, nc));
    k_chunk_build<<<nc, CH_T, 0, s>>>(cp.c_graph, cp.c_n0, cp.c_own, p->loc_ptr, p->nbr_ptr, p->nbr_off, p->nbr, 0,
                                      cp.c_need_n, adj_n, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                      p->d_status);
    DDG_LAUNCH_CHECK();
    std::vector<int> hn(nc), ha(nc);
    DDG_CU(cudaMemcpyAsync(hn.data(), cp.c_need_n, sizeof(int) * nc, cudaMemcpyDeviceToHost, s));
    DDG_CU(cudaMemcpyAsync(ha.data(), adj_n, sizeof(int) * nc, cudaMemcpyDeviceToHost, s));
    DDG_CU(cudaStreamSynchronize(s));
    DDG_TRY(check_status(p, "GNN chunks"));
    std::vector<int> noff(nc), aoff(nc), abase(nc);
    long long tn = 0, ta = 0, tp = 0;
    int maxn = 0;
    for (int q = 0; q < nc; ++q) {
        noff[q] = (int)tn;
        abase[q] = (int)ta;
        aoff[q] = (int)tp;
        tn += hn[q];
        ta += ha[q];
        tp += cown[q] + 1;
        maxn = std::max(maxn, hn[q]);
    }
    cp.max_need = maxn;
    DDG_TRY(dalloc(c, cp.allocs, &cp.need, tn));
    DDG_TRY(dalloc(c, cp.allocs, &cp.adj, ta));
    DDG_TRY(dalloc(c, cp.allocs, &cp.adj_ptr, tp));
    DDG_CU(cudaMemcpyAsync(cp.c_need_off, noff.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    DDG_CU(cudaMemcpyAsync(cp.c_adj_off, aoff.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    DDG_CU(cudaMemcpyAsync(cp.c_adj_base, abase.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    k_chunk_build<<<nc, CH_T, 0, s>>>(cp.c_graph, cp.c_n0, cp.c_own, p->loc_ptr, p->nbr_ptr, p->nbr_off, p->nbr, 1,
                                      nullptr, nullptr, cp.c_need_off, cp.need, cp.c_adj_off, cp.adj_ptr,
                                      cp.c_adj_base, cp.adj, p->d_status);
    DDG_LAUNCH_CHECK();
    DDG_CU(sc.drop(adj_n));
    DDG_CU(cudaStreamSynchronize(s));
    return check_status(p, "GNN chunks");
}

template <int T>
static int32_t launch_chunks(ddg_problem *p, const ChunkArgs &base, cudaStream_t s) {
    static bool configured = false;
    if (!configured) {
        DDG_CU(cudaFuncSetAttribute(k_dss_chunk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        configured = true;
    }
    const ddg_model *m = p->model;
    const size_t smem = (size_t)p->chunk.max_need * 2 * D * sizeof(float);
    for (int blk = 0; blk < m->kbar; ++blk) {
        ChunkArgs a = base;
        a.first = blk == 0;
        a.last = blk == m->kbar - 1;
        a.h_in = (blk & 1) ? p->dss_h2 : p->dss_h;
        a.h_out = (blk & 1) ? p->dss_h : p->dss_h2;
        const BlockWeights *W = reinterpret_cast<const BlockWeights *>(w_packed_host(p)) + blk;
        k_dss_chunk<T><<<p->chunk.nchunks, T, smem, s>>>(*W, a);
    }
    DDG_LAUNCHES(m->kbar);
    return DDG_OK;
}

template <int T>
static int32_t fused_configure() {
    static bool configured = false;
    if (!configured) {
        DDG_CU(cudaFuncSetAttribute(k_dss_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        configured = true;
    }
    return DDG_OK;
}

template <int T>
static int32_t fused_ctas_per_sm(size_t smem, int *out) {
    DDG_TRY(fused_configure<T>());
    DDG_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_dss_fused<T>, T, smem));
    return DDG_OK;
}

// Global chunk plan of schedules 3 and 4: the concatenated graphs' nodes cut into
// equal-work ranges, as many as fill every SM's resident CTAs a whole number of
// times, so every SM gets the same work per block.  Schedule 3 (tc = false) takes
// at most 2T own nodes per chunk; schedule 4 (tc = true) at most T own nodes and
// TC_NEED needed nodes (own plus outside neighbours), splitting any range whose
// needed nodes exceed that in two until none does.
int32_t chunk_build_global(ddg_problem *p, int T, bool tc) {
    ddg_ctx *c = p->ctx;
    cudaStream_t s = p->stream;
    chunk_free(p);
    ChunkPlan &cp = p->chunk;
    const long long n = p->sum_loc;
    const int K = p->K;
    int sms = 0, per_sm = 0;
    DDG_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    const long long own_cap = tc ? T : 2LL * T;
    if (tc) {
        if (T != TC_T) {
            set_error("schedule-4 chunk width must be 256");
            return DDG_INVALID_ARG;
        }
        DDG_TRY(tc_ctas_per_sm(&per_sm));
        per_sm = TC_CTAS_PER_SM;  // the launch's grid (dss_tc_launch)
    } else {
        const size_t smem_est = fused_smem(3 * T, 2 * T);  // 2T own + T outside nodes
        switch (T) {
            case 128: DDG_TRY(fused_ctas_per_sm<128>(smem_est, &per_sm)); break;
            case 256: DDG_TRY(fused_ctas_per_sm<256>(smem_est, &per_sm)); break;
            default: set_error("schedule-3 chunk width must be 128 or 256"); return DDG_INVALID_ARG;
        }
    }
    const long long slots = (long long)sms * std::max(1, per_sm);
    const long long waves = std::max(1LL, (n + slots * own_cap - 1) / (slots * own_cap));
    // at least half the cap: a small problem takes fewer CTAs (and leaves SMs to the kernels of
    // other streams) rather than slivers of a few nodes with large halos
    const long long cs = std::max<long long>(own_cap / 2, (n + slots * waves - 1) / (slots * waves));
    const long long nc_target = (n + cs - 1) / cs;
    std::vector<int> lp(K + 1), lk(K), nptr(n + K), gid(n), cn0, cown;
    DDG_CU(cudaMemcpyAsync(lp.data(), p->loc_ptr, sizeof(int) * (K + 1), cudaMemcpyDeviceToHost, s));
    DDG_CU(cudaMemcpyAsync(lk.data(), p->loc_nint, sizeof(int) * K, cudaMemcpyDeviceToHost, s));
    DDG_CU(cudaMemcpyAsync(nptr.data(), p->nbr_ptr, sizeof(int) * (n + K), cudaMemcpyDeviceToHost, s));
    DDG_CU(cudaStreamSynchronize(s));
    // estimated instructions of a node in one block: projections and node MLPs, plus per
    // neighbour the edge geometry and the out-message, and the in-message for unknowns
    std::vector<double> work(n);
    double total = 0.0;
    for (int g = 0; g < K; ++g)
        for (int u = lp[g]; u < lp[g + 1]; ++u) {
            gid[u] = g;
            const int j = u - lp[g];
            const int deg = nptr[lp[g] + g + j + 1] - nptr[lp[g] + g + j];
            work[u] = 500.0 + (j < lk[g] ? 95.0 : 60.0) * deg;
            total += work[u];
        }
    // equal-work ranges (at most own_cap nodes each), about nc_target of them
    const double per = total / (double)nc_target;
    double acc = 0.0;
    long long start = 0;
    for (long long u = 0; u < n; ++u) {
        acc += work[u];
        const long long len = u + 1 - start;
        if (len == own_cap || acc >= per * (double)(cn0.size() + 1) || u == n - 1) {
            cn0.push_back((int)start);
            cown.push_back((int)len);
            start = u + 1;
        }
    }
    DDG_TRY(dalloc(c, cp.allocs, &cp.gid, n));
    DDG_CU(cudaMemcpyAsync(cp.gid, gid.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    // pass 0: needed nodes and adjacency entries per chunk (schedule 4: split the ranges whose
    // needed nodes exceed the cap, and count again)
    std::vector<int> hn, ha;
    Scratch sc(s);
    for (int round = 0;; ++round) {
        const int nc = (int)cn0.size();
        int *t_n0 = nullptr, *t_own = nullptr, *t_need = nullptr, *t_adj = nullptr;
        DDG_CU(sc.get(&t_n0, nc));
        DDG_CU(sc.get(&t_own, nc));
        DDG_CU(sc.get(&t_need, nc));
        DDG_CU(sc.get(&t_adj, nc));
        DDG_CU(cudaMemcpyAsync(t_n0, cn0.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
        DDG_CU(cudaMemcpyAsync(t_own, cown.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
        k_gchunk_build<<<nc, 256, 0, s>>>(t_n0, t_own, cp.gid, p->loc_ptr, p->loc_nint, p->nbr_ptr, p->nbr_off,
                                          p->nbr, p->sub_ptr, p->sub_idx, 0, t_need, t_adj, nullptr, nullptr,
                                          nullptr, nullptr, nullptr, nullptr, nullptr, p->loc_xy, nullptr,
                                          p->d_status);
        DDG_LAUNCH_CHECK();
        hn.assign(nc, 0);
        ha.assign(nc, 0);
        DDG_CU(cudaMemcpyAsync(hn.data(), t_need, sizeof(int) * nc, cudaMemcpyDeviceToHost, s));
        DDG_CU(cudaMemcpyAsync(ha.data(), t_adj, sizeof(int) * nc, cudaMemcpyDeviceToHost, s));
        DDG_CU(cudaStreamSynchronize(s));
        DDG_TRY(check_status(p, "GNN chunks"));
        for (void *q : {(void *)t_n0, (void *)t_own, (void *)t_need, (void *)t_adj}) DDG_CU(sc.drop(q));
        if (!tc) break;
        std::vector<int> n0b, ownb;
        bool split = false;
        for (int q = 0; q < nc; ++q) {
            if (hn[q] > TC_NEED && cown[q] > 1) {
                const int h1 = cown[q] / 2;
                n0b.push_back(cn0[q]);
                ownb.push_back(h1);
                n0b.push_back(cn0[q] + h1);
                ownb.push_back(cown[q] - h1);
                split = true;
            } else {
                n0b.push_back(cn0[q]);
                ownb.push_back(cown[q]);
            }
        }
        if (!split) break;
        if (round == 8) {
            set_error("a schedule-4 GNN chunk keeps more needed nodes than a CTA holds");
            return DDG_TOO_LARGE;
        }
        cn0.swap(n0b);
        cown.swap(ownb);
    }
    const int nc = (int)cn0.size();
    cp.T = T;
    cp.global = true;
    cp.tc = tc;
    cp.nchunks = nc;
    DDG_TRY(dalloc(c, cp.allocs, &cp.info, n));
    DDG_TRY(dalloc(c, cp.allocs, &cp.c_n0, nc));
    DDG_TRY(dalloc(c, cp.allocs, &cp.c_own, nc));
    DDG_TRY(dalloc(c, cp.allocs, &cp.c_need_off, nc));
    DDG_TRY(dalloc(c, cp.allocs, &cp.c_need_n, nc));
    DDG_TRY(dalloc(c, cp.allocs, &cp.c_adj_off, nc));
    DDG_TRY(dalloc(c, cp.allocs, &cp.c_adj_base, nc));
    DDG_CU(cudaMemcpyAsync(cp.c_n0, cn0.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    DDG_CU(cudaMemcpyAsync(cp.c_own, cown.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    DDG_CU(cudaMemcpyAsync(cp.c_need_n, hn.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    std::vector<int> noff(nc), aoff(nc), abase(nc);
    long long tn = 0, ta = 0, tp = 0;
    int maxn = 0;
    size_t max_smem = 0;
    for (int q = 0; q < nc; ++q) {
        noff[q] = (int)tn;
        abase[q] = (int)ta;
        aoff[q] = (int)tp;
        tn += hn[q];
        ta += ha[q];
        tp += cown[q] + 1;
        maxn = std::max(maxn, hn[q]);
        max_smem = std::max(max_smem, tc ? (size_t)TC_SMEM : fused_smem(hn[q], cown[q]));
    }
    cp.max_need = maxn;
    cp.max_smem = max_smem;
    if (max_smem > 227 * 1024) {
        set_error("a GNN chunk needs more shared memory than a CTA has");
        return DDG_TOO_LARGE;
    }
    DDG_TRY(dalloc(c, cp.allocs, &cp.need, tn));
    DDG_TRY(dalloc(c, cp.allocs, &cp.adj, ta));
    DDG_TRY(dalloc(c, cp.allocs, &cp.adjx, ta));
    DDG_TRY(dalloc(c, cp.allocs, &cp.adj_ptr, tp));
    DDG_CU(cudaMemcpyAsync(cp.c_need_off, noff.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    DDG_CU(cudaMemcpyAsync(cp.c_adj_off, aoff.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    DDG_CU(cudaMemcpyAsync(cp.c_adj_base, abase.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    k_gchunk_build<<<nc, 256, 0, s>>>(cp.c_n0, cp.c_own, cp.gid, p->loc_ptr, p->loc_nint, p->nbr_ptr, p->nbr_off,
                                      p->nbr, p->sub_ptr, p->sub_idx, 1, nullptr, nullptr, cp.c_need_off, cp.need,
                                      cp.c_adj_off, cp.adj_ptr, cp.c_adj_base, cp.adj, cp.info, p->loc_xy, cp.adjx,
                                      p->d_status);
    DDG_LAUNCH_CHECK();
    DDG_CU(cudaStreamSynchronize(s));
    return check_status(p, "GNN chunks");
}

template <int T>
static int32_t launch_fused(ddg_problem *p, const ChunkArgs &base, cudaStream_t s) {
    DDG_TRY(fused_configure<T>());
    const ddg_model *m = p->model;
    const size_t smem = p->chunk.max_smem;
    for (int blk = 0; blk < m->kbar; ++blk) {
        ChunkArgs a = base;
        a.first = blk == 0;
        a.last = blk == m->kbar - 1;
        a.h_in = (blk & 1) ? p->dss_h2 : p->dss_h;
        a.h_out = (blk & 1) ? p->dss_h : p->dss_h2;
        const FusedWeights *W = reinterpret_cast<const FusedWeights *>(w_fused_host(p)) + blk;
        // programmatic dependent launch: block blk+1's CTAs are scheduled as block blk's CTAs
        // retire, hiding the launch gap between the 30 launches of an application
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(p->chunk.nchunks);
        cfg.blockDim = dim3(T);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = p->ctx->pdl ? 1 : 0;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        DDG_CU(cudaLaunchKernelEx(&cfg, k_dss_fused<T>, *W, a));
    }
    DDG_LAUNCHES(m->kbar);
    return DDG_OK;
}

static ChunkArgs chunk_args(ddg_problem *p, const double *r, const int *stop) {
    const ChunkPlan &cp = p->chunk;
    ChunkArgs a{};
    a.c_graph = cp.c_graph;
    a.c_n0 = cp.c_n0;
    a.c_own = cp.c_own;
    a.c_need_off = cp.c_need_off;
    a.c_need_n = cp.c_need_n;
    a.need = cp.need;
    a.c_adj_off = cp.c_adj_off;
    a.adj_ptr = cp.adj_ptr;
    a.adj = cp.adj;
    a.adjx = cp.adjx;
    a.c_adj_base = cp.c_adj_base;
    a.loc_ptr = p->loc_ptr;
    a.loc_nint = p->loc_nint;
    a.gid = cp.gid;
    a.info = cp.info;
    a.sub_ptr = p->sub_ptr;
    a.sub_idx = p->sub_idx;
    a.loc_xy = p->loc_xy;
    a.r = r;
    a.s = p->s;
    a.corr = p->corr;
    a.c = p->dss_c;
    a.n_total = p->sum_loc;
    a.alpha = p->model->alpha;
    a.stop = stop;
    a.status = p->d_status;
    a.h_in = p->dss_h;
    a.h_out = p->dss_h2;
    return a;
}

int32_t dss_chunk_launch(ddg_problem *p, const double *r, const int *stop, cudaStream_t s) {
    const ChunkPlan &cp = p->chunk;
    const ChunkArgs a = chunk_args(p, r, stop);
    if (p->dss_sched == 5) return dss_d_launch(p, a, s);
    if (p->dss_sched == 6)
        return dss_mma_launch(p, a, w_fused_host(p), p->w_bf16 ? p->bf16_mma_dev : p->model->mma_w, s);
    if (cp.tc) return dss_tc_launch(p, a, w_fused_host(p), p->w_bf16 ? p->bf16_tc_dev : p->model->tc_w, s);
    if (cp.global) {
        switch (cp.T) {
            case 128: return launch_fused<128>(p, a, s);
            case 256: return launch_fused<256>(p, a, s);
            default: set_error("no chunk plan"); return DDG_INVALID_ARG;
        }
    }
    switch (cp.T) {
        case 128: return launch_chunks<128>(p, a, s);
        case 192: return launch_chunks<192>(p, a, s);
        case 256: return launch_chunks<256>(p, a, s);
        default: set_error("no chunk plan"); return DDG_INVALID_ARG;
    }
}

// ---------------------------------------------------------------- fused step over several problems
template <int T>
static int32_t launch_group(ddg_problem *const *ps, int n, const int *cpre, const ChunkArgs *dev_args,
                            size_t smem, cudaStream_t s) {
    static bool configured = false;
    if (!configured) {
        DDG_CU(cudaFuncSetAttribute(k_dss_fused_group<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    227 * 1024));
        configured = true;
    }
    const ddg_model *m = ps[0]->model;
    for (int blk = 0; blk < m->kbar; ++blk) {
        GroupArgs g{};
        g.n = n;
        g.first = blk == 0;
        g.last = blk == m->kbar - 1;
        g.odd = blk & 1;
        for (int i = 0; i <= n; ++i) g.cpre[i] = cpre[i];
        g.args = dev_args;
        const FusedWeights *W = reinterpret_cast<const FusedWeights *>(w_fused_host(ps[0])) + blk;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cpre[n]);
        cfg.blockDim = dim3(T);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = ps[0]->ctx->pdl ? 1 : 0;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        DDG_CU(cudaLaunchKernelEx(&cfg, k_dss_fused_group<T>, *W, g));
    }
    DDG_LAUNCHES(m->kbar);
    return DDG_OK;
}

bool dss_group_compatible(const ddg_problem *a, const ddg_problem *b) {
    return a->kind == DDG_DDM_GNN && b->kind == DDG_DDM_GNN && a->model == b->model && a->w_bf16 == b->w_bf16 &&
           a->dss_sched == 3 && b->dss_sched == 3 && a->chunk.T == b->chunk.T;
}

int32_t dss_group_prepare(ddg_problem *p) {
    if (p->kind != DDG_DDM_GNN) return DDG_INVALID_ARG;
    if (p->model->d != DSS_D) return DDG_TOO_LARGE;  // fused group steps run schedule 3 (d = 10 only)
    if (p->dss_sched != 3 || p->chunk.T != GROUP_T || !p->chunk.global || p->chunk.tc) {
        DDG_TRY(chunk_build_global(p, GROUP_T, false));
        p->dss_sched = 3;
    }
    return DDG_OK;
}

int32_t dss_group_launch(ddg_problem *const *ps, const double *const *rs, const int *const *stops, int n,
                         ChunkArgs *dev_args, bool upload, cudaStream_t s) {
    if (n < 1 || n > MAX_GROUP) {
        set_error("a fused GNN step takes 1 to 32 problems");
        return DDG_INVALID_ARG;
    }
    int cpre[MAX_GROUP + 1];
    size_t smem = 0;
    cpre[0] = 0;
    std::vector<ChunkArgs> host(n);
    for (int i = 0; i < n; ++i) {
        if (!dss_group_compatible(ps[0], ps[i])) {
            set_error("problems of one fused GNN step must share model, weights precision and chunk plan width");
            return DDG_INVALID_ARG;
        }
        host[i] = chunk_args(ps[i], rs[i], stops[i]);
        cpre[i + 1] = cpre[i] + ps[i]->chunk.nchunks;
        smem = std::max(smem, ps[i]->chunk.max_smem);
    }
    if (upload)
        DDG_CU(cudaMemcpyAsync(dev_args, host.data(), sizeof(ChunkArgs) * n, cudaMemcpyHostToDevice, s));
    switch (ps[0]->chunk.T) {
        case 128: return launch_group<128>(ps, n, cpre, dev_args, smem, s);
        case 256: return launch_group<256>(ps, n, cpre, dev_args, smem, s);
        default: set_error("no chunk plan"); return DDG_INVALID_ARG;
    }
}

size_t dss_group_args_bytes() { return sizeof(ChunkArgs) * MAX_GROUP; }

static size_t dss_smem_bytes(int nmax, int emax) {
    size_t b = 128 + 2 * (size_t)BLOCK_BYTES;
    b += (size_t)nmax * 2 * D * sizeof(float);
    b += (size_t)nmax * sizeof(float2);
    b += (size_t)((nmax + 1 + 7) & ~7) * sizeof(uint16_t);
    b += (size_t)emax * sizeof(uint16_t);
    return (b + 127) & ~(size_t)127;
}

template <int P>
static int32_t launch_p(const DssArgs &a, int K, size_t smem, cudaStream_t s) {
    static bool configured = false;
    if (!configured) {
        DDG_CU(cudaFuncSetAttribute(k_dss<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        configured = true;
    }
    k_dss<P><<<K, DSS_THREADS, smem, s>>>(a);
    DDG_LAUNCH_CHECK();
    return DDG_OK;
}

template <int P>
static int32_t launch_steps(ddg_problem *p, const DssStepArgs &base, size_t smem, cudaStream_t s) {
    static bool configured = false;
    if (!configured) {
        DDG_CU(cudaFuncSetAttribute(k_dss_step<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        configured = true;
    }
    const ddg_model *m = p->model;
    for (int blk = 0; blk < m->kbar; ++blk) {
        DssStepArgs a = base;
        a.first = blk == 0;
        a.last = blk == m->kbar - 1;
        const BlockWeights *W = reinterpret_cast<const BlockWeights *>(w_packed_host(p)) + blk;
        k_dss_step<P><<<p->K, DSS_THREADS, smem, s>>>(*W, a);
    }
    DDG_LAUNCHES(m->kbar);
    return DDG_OK;
}

int32_t dss_step_launch(ddg_problem *p, const double *r, const int *stop, cudaStream_t s) {
    DssStepArgs a;
    a.order = p->lpt_order;
    a.loc_ptr = p->loc_ptr;
    a.loc_nint = p->loc_nint;
    a.nbr_ptr = p->nbr_ptr;
    a.nbr_off = p->nbr_off;
    a.sub_ptr = p->sub_ptr;
    a.sub_idx = p->sub_idx;
    a.nbr = p->nbr;
    a.loc_xy = p->loc_xy;
    a.r = r;
    a.s = p->s;
    a.corr = p->corr;
    a.h = p->dss_h;
    a.c = p->dss_c;
    a.n_total = p->sum_loc;
    a.alpha = p->model->alpha;
    a.first = a.last = 0;
    a.stop = stop;
    size_t smem = (size_t)p->max_loc * 2 * D * sizeof(float);
    switch (cdiv(p->max_loc, DSS_THREADS)) {
        case 1: return launch_steps<1>(p, a, smem, s);
        case 2: return launch_steps<2>(p, a, smem, s);
        case 3: return launch_steps<3>(p, a, smem, s);
        case 4: return launch_steps<4>(p, a, smem, s);
        default: set_error("local graph too large for the GNN kernel"); return DDG_TOO_LARGE;
    }
}

int32_t dss_launch_args(ddg_problem *p, const double *r, const int *stop, cudaStream_t s) {
    if (p->dss_sched == 1) return dss_step_launch(p, r, stop, s);
    if (p->dss_sched >= 2) return dss_chunk_launch(p, r, stop, s);
    const ddg_model *m = p->model;
    DssArgs a;
    a.weights = w_packed_dev(p);
    a.kbar = m->kbar;
    a.alpha = m->alpha;
    a.order = p->lpt_order;
    a.loc_ptr = p->loc_ptr;
    a.loc_nint = p->loc_nint;
    a.nbr_ptr = p->nbr_ptr;
    a.nbr_off = p->nbr_off;
    a.sub_ptr = p->sub_ptr;
    a.sub_idx = p->sub_idx;
    a.nbr = p->nbr;
    a.loc_xy = p->loc_xy;
    a.r = r;
    a.s = p->s;
    a.corr = p->corr;
    a.nmax = p->max_loc;
    a.emax = p->max_edges;
    a.stop = stop;
    a.status = p->d_status;
    a.test_skip_copy = getenv("DDG_TEST_WAIT_TIMEOUT") != nullptr;  // failure test only
    size_t smem = dss_smem_bytes(a.nmax, a.emax);
    int P = cdiv(p->max_loc, DSS_THREADS);
    switch (P) {
        case 1: return launch_p<1>(a, p->K, smem, s);
        case 2: return launch_p<2>(a, p->K, smem, s);
        case 3: return launch_p<3>(a, p->K, smem, s);
        case 4: return launch_p<4>(a, p->K, smem, s);
        default: set_error("local graph too large for the GNN kernel"); return DDG_TOO_LARGE;
    }
}

// Schedules 0 and 1 hold a whole local graph in one CTA's shared memory (at most
// DSS_MAX_NODES nodes); the chunked schedules 2 and 3 take graphs up to the
// 16-bit local ids' limit, e.g. the paper's sub-meshes of 2,000 nodes with overlap.
int32_t dss_check_capacity(ddg_problem *p) {
    if (p->max_loc > 65535) {
        set_error("local graph of " + std::to_string(p->max_loc) + " nodes exceeds the 65,535 nodes of 16-bit local ids");
        return DDG_TOO_LARGE;
    }
    p->dss_whole_graph = p->max_loc <= DSS_MAX_NODES && p->max_edges <= 65535 &&
                         dss_smem_bytes(p->max_loc, p->max_edges) <= 227 * 1024;
    return DDG_OK;
}

}  // namespace ddg
