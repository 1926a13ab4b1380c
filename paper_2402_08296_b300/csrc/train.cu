// Training of the DSS local solver on the decomposition's own local problems
// (Section III-B, Eq. 23; optimiser of Section IV-B), with hand-written
// forward and backward kernels.
//
// Samples: the normalised restricted residuals c = R_i r^n / |R_i r^n| of the
// iterations of a DDM-LU preconditioned CG run on the problem (Section IV-A's
// recipe), each paired with its local graph G_i and local matrix R_i A R_i^T.
// Loss per sample: sum over blocks k of L_res(r_hat^k) = mean_t ((A_i r_hat^k - c)_t^2)
// (Eqs. 11, 23); a step averages it over the batch.
//
// Kernels (one CTA per sample):
//  k_tr_fwd  the inference of k_dss, saving h^k after every block and the
//            decoded r_hat^k of every block;
//  k_tr_bwd  the loss, its gradient through the local matrix, then the blocks in
//            reverse: decoder, Psi, the two second layers, the edge messages
//            (recomputed from the saved h^k) and the node projections. The
//            gradient of a neighbour projection is gathered at its owner, so no
//            scatter is needed; weight gradients are reduced over a warp, added
//            in shared memory and flushed once per block with global atomics.
//  k_tr_norm / k_tr_adam  global-norm clipping and Adam on the flat weights,
//            then repacking into the inference layout.
#include "dss_layout.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace ddg {

constexpr int TR_T = 256;

struct TrainArgs {
    const float *W;            // packed weights, kbar blocks
    int kbar;
    float alpha;
    int B;                     // samples in the batch
    const int *graph;          // [B] local graph of each sample
    const double *const *res;  // [B] global residual vector of each sample (n_free)
    const int *nbase;          // [B+1] offset of each sample's nodes in the scratch arrays
    const int *kbase;          // [B+1] offset of each sample's unknowns
    long long NB, NK;          // total nodes / unknowns of the batch
    const int *loc_ptr, *loc_nint, *nbr_ptr, *nbr_off, *sub_ptr, *sub_idx;
    const uint16_t *nbr;
    const float2 *loc_xy;
    const int *lm_ptr;         // local matrices: per graph CSR over unknowns (graph i's rows at lm_row[i])
    const int *lm_row;         // [K+1] first row pointer of each graph inside lm_ptr
    const uint16_t *lm_col;
    const float *lm_val;
    float *c;                  // [NB]
    float *hsave;              // [(kbar+1) * D][NB]
    float *rhat;               // [kbar][NK]
    float *ghat;               // [kbar][NK]   dL / d r_hat^k
    float *res_k;              // [NK]          A r_hat - c of the current block
    float *scr;                // [8 * D][NB]   Pa_o, Pa_i, Pb_o, Pb_i, dS_o, dS_i, dh, dh_new
    float *gpack;              // [kbar][BLOCK_FLOATS] weight gradients, packed layout
    float *loss;               // [B]
};

enum { SC_PAO = 0, SC_PAI = 1, SC_PBO = 2, SC_PBI = 3, SC_DSO = 4, SC_DSI = 5, SC_DH = 6 };

__device__ __forceinline__ float *scv(const TrainArgs &a, int which, int o, long long node) {
    return a.scr + ((long long)which * D + o) * a.NB + node;
}

__device__ __forceinline__ float warp_sum_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// gsh[idx] += sum over the warp of v (every lane of the warp must call)
__device__ __forceinline__ void gacc(float *gsh, int idx, float v) {
    v = warp_sum_f(v);
    if ((threadIdx.x & 31) == 0 && v != 0.f) atomicAdd(&gsh[idx], v);
}

// ---------------------------------------------------------------- forward with saved states
__global__ void __launch_bounds__(TR_T) k_tr_fwd(TrainArgs a) {
    __shared__ __align__(16) float Wsh[BLOCK_FLOATS];
    __shared__ double red[32];
    const int b = blockIdx.x, g = a.graph[b];
    const int lp = a.loc_ptr[g], nl = a.loc_ptr[g + 1] - lp, k = a.loc_nint[g];
    const int s0 = a.sub_ptr[g];
    const long long nb0 = a.nbase[b], kb0 = a.kbase[b];
    const int *gptr = a.nbr_ptr + lp + g;
    const uint16_t *gn = a.nbr + a.nbr_off[g];
    const float2 *xy = a.loc_xy + lp;
    const double *res = a.res[b];
    double ss = 0.0;
    for (int t = threadIdx.x; t < k; t += TR_T) {
        double v = res[a.sub_idx[s0 + t]];
        ss += v * v;
    }
    ss = block_sum(ss, red);
    if (threadIdx.x == 0) red[31] = ss;
    __syncthreads();
    const double s = sqrt(red[31]);
    for (int j = threadIdx.x; j < nl; j += TR_T) {
        float cj = (j < k && s > 0.0) ? (float)(res[a.sub_idx[s0 + j]] / s) : 0.f;
        a.c[nb0 + j] = cj;
        for (int o = 0; o < D; ++o) a.hsave[(long long)o * a.NB + nb0 + j] = 0.f;
    }
    float *Pb = a.scr + (long long)SC_PBO * D * a.NB;  // reuse scratch rows: [2D][NB] as Pb_o|Pb_i
    for (int blk = 0; blk < a.kbar; ++blk) {
        __syncthreads();
        for (int q = threadIdx.x; q < BLOCK_FLOATS; q += TR_T) Wsh[q] = a.W[(size_t)blk * BLOCK_FLOATS + q];
        __syncthreads();
        const float *hin = a.hsave + (long long)blk * D * a.NB;
        float *hout = a.hsave + (long long)(blk + 1) * D * a.NB;
        for (int j = threadIdx.x; j < nl; j += TR_T) {
            float h[D], po[D], pi[D];
            for (int o = 0; o < D; ++o) { h[o] = hin[(long long)o * a.NB + nb0 + j]; po[o] = 0.f; pi[o] = 0.f; }
            mv_acc<D>(po, Wsh + OFF_OUT + PHI_WB, h);
            mv_acc<D>(pi, Wsh + OFF_IN + PHI_WB, h);
            for (int o = 0; o < D; ++o) {
                Pb[(long long)o * a.NB + nb0 + j] = po[o];
                Pb[(long long)(D + o) * a.NB + nb0 + j] = pi[o];
            }
        }
        __syncthreads();
        for (int j = threadIdx.x; j < nl; j += TR_T) {
            const bool inner = j < k;
            float h[D], Pao[D], Pai[D], So[D], Si[D];
            for (int o = 0; o < D; ++o) { h[o] = hin[(long long)o * a.NB + nb0 + j]; So[o] = 0.f; Si[o] = 0.f; }
            load_vec(Pao, Wsh + OFF_OUT + PHI_B1);
            load_vec(Pai, Wsh + OFF_IN + PHI_B1);
            mv_acc<D>(Pao, Wsh + OFF_OUT + PHI_WA, h);
            mv_acc<D>(Pai, Wsh + OFF_IN + PHI_WA, h);
            const float2 xj = xy[j];
            int dout = 0, din = 0;
            for (int e = gptr[j]; e < gptr[j + 1]; ++e) {
                const int l = gn[e];
                const float2 xl = xy[l];
                const float dx = xl.x - xj.x, dy = xl.y - xj.y, dn = sqrtf(dx * dx + dy * dy);
                float pbo[D], pbi[D];
                for (int o = 0; o < D; ++o) {
                    pbo[o] = Pb[(long long)o * a.NB + nb0 + l];
                    pbi[o] = Pb[(long long)(D + o) * a.NB + nb0 + l];
                }
                if (l < k) { edge_msg(So, Pao, pbo, Wsh + OFF_OUT + PHI_WE, dx, dy, dn); ++dout; }
                if (inner) { edge_msg(Si, Pai, pbi, Wsh + OFF_IN + PHI_WE, -dx, -dy, dn); ++din; }
            }
            float fo[D], fi[D];
            for (int o = 0; o < D; ++o) {
                fo[o] = dout * Wsh[OFF_OUT + PHI_B2 + o];
                fi[o] = din * Wsh[OFF_IN + PHI_B2 + o];
            }
            mv_acc<D>(fo, Wsh + OFF_OUT + PHI_W2, So);
            mv_acc<D>(fi, Wsh + OFF_IN + PHI_W2, Si);
            float hid[D];
            load_vec(hid, Wsh + OFF_PSI + PSI_B1);
            mv_acc<D>(hid, Wsh + OFF_PSI + PSI_W1, h);
            float cc[1] = {a.c[nb0 + j]};
            mv_acc<1>(hid, Wsh + OFF_PSI + PSI_W1 + D * DP, cc);
            mv_acc<D>(hid, Wsh + OFF_PSI + PSI_W1 + (D + 1) * DP, fo);
            mv_acc<D>(hid, Wsh + OFF_PSI + PSI_W1 + (2 * D + 1) * DP, fi);
            for (int o = 0; o < D; ++o) hid[o] = relu(hid[o]);
            float out[D];
            load_vec(out, Wsh + OFF_PSI + PSI_B2);
            mv_acc<D>(out, Wsh + OFF_PSI + PSI_W2, hid);
            for (int o = 0; o < D; ++o) {
                h[o] = fmaf(a.alpha, out[o], h[o]);
                hout[(long long)o * a.NB + nb0 + j] = h[o];
            }
            if (inner) {
                float dh[D];
                load_vec(dh, Wsh + OFF_DEC + DEC_B1);
                mv_acc<D>(dh, Wsh + OFF_DEC + DEC_W1, h);
                float y = Wsh[OFF_DEC + DEC_B2];
                for (int o = 0; o < D; ++o) y = fmaf(Wsh[OFF_DEC + DEC_W2 + o], relu(dh[o]), y);
                a.rhat[(long long)blk * a.NK + kb0 + j] = y;
            }
        }
    }
}

// ---------------------------------------------------------------- loss and backward
__global__ void __launch_bounds__(TR_T) k_tr_bwd(TrainArgs a) {
    __shared__ __align__(16) float Wsh[BLOCK_FLOATS];
    __shared__ float gsh[BLOCK_FLOATS];
    __shared__ double red[32];
    const int b = blockIdx.x, g = a.graph[b];
    const int lp = a.loc_ptr[g], nl = a.loc_ptr[g + 1] - lp, k = a.loc_nint[g];
    const long long nb0 = a.nbase[b], kb0 = a.kbase[b];
    const int *gptr = a.nbr_ptr + lp + g;
    const uint16_t *gn = a.nbr + a.nbr_off[g];
    const float2 *xy = a.loc_xy + lp;
    const int *lmp = a.lm_ptr + a.lm_row[g];  // k + 1 row pointers
    const int lm0 = lmp[0];
    const float gscale = 2.f / ((float)k * (float)a.B);
    // loss sum_k mean (A r_hat^k - c)^2 and its gradient 2/(k B) A (A r_hat^k - c)
    double lsum = 0.0;
    for (int blk = 0; blk < a.kbar; ++blk) {
        const float *rh = a.rhat + (long long)blk * a.NK + kb0;
        for (int t = threadIdx.x; t < k; t += TR_T) {
            float acc = 0.f;
            for (int e = lmp[t]; e < lmp[t + 1]; ++e) acc += a.lm_val[e] * rh[a.lm_col[e]];
            float rr = acc - a.c[nb0 + t];
            a.res_k[kb0 + t] = rr;
            lsum += (double)rr * rr;
        }
        __syncthreads();
        float *gh = a.ghat + (long long)blk * a.NK + kb0;
        for (int t = threadIdx.x; t < k; t += TR_T) {
            float acc = 0.f;
            for (int e = lmp[t]; e < lmp[t + 1]; ++e) acc += a.lm_val[e] * a.res_k[kb0 + a.lm_col[e]];
            gh[t] = gscale * acc;
        }
        __syncthreads();
    }
    (void)lm0;
    lsum = block_sum(lsum, red);
    if (threadIdx.x == 0) a.loss[b] = (float)(lsum / k);
    for (int j = threadIdx.x; j < nl; j += TR_T)
        for (int o = 0; o < D; ++o) *scv(a, SC_DH, o, nb0 + j) = 0.f;

    const int n_pass = (nl + TR_T - 1) / TR_T;
    for (int blk = a.kbar - 1; blk >= 0; --blk) {
        __syncthreads();
        for (int q = threadIdx.x; q < BLOCK_FLOATS; q += TR_T) {
            Wsh[q] = a.W[(size_t)blk * BLOCK_FLOATS + q];
            gsh[q] = 0.f;
        }
        __syncthreads();
        const float *h0 = a.hsave + (long long)blk * D * a.NB;
        const float *h1 = a.hsave + (long long)(blk + 1) * D * a.NB;
        // (a) decoder of block blk, and the neighbour-side projections of the forward recomputation
        for (int pass = 0; pass < n_pass; ++pass) {
            const int j = pass * TR_T + threadIdx.x;
            const bool act = j < nl;
            const bool inner = j < k;
            float h[D], u[D], gy = 0.f;
            for (int o = 0; o < D; ++o) h[o] = act ? h1[(long long)o * a.NB + nb0 + j] : 0.f;
            load_vec(u, Wsh + OFF_DEC + DEC_B1);
            mv_acc<D>(u, Wsh + OFF_DEC + DEC_W1, h);
            if (inner) gy = a.ghat[(long long)blk * a.NK + kb0 + j];
            float du[D];
            for (int o = 0; o < D; ++o) {
                gacc(gsh, OFF_DEC + DEC_W2 + o, gy * relu(u[o]));
                du[o] = u[o] > 0.f ? gy * Wsh[OFF_DEC + DEC_W2 + o] : 0.f;
                gacc(gsh, OFF_DEC + DEC_B1 + o, du[o]);
            }
            gacc(gsh, OFF_DEC + DEC_B2, gy);
            for (int i = 0; i < D; ++i)
                for (int o = 0; o < D; ++o) gacc(gsh, OFF_DEC + DEC_W1 + i * DP + o, du[o] * h[i]);
            if (act) {
                for (int i = 0; i < D; ++i) {
                    float v = 0.f;
                    for (int o = 0; o < D; ++o) v += Wsh[OFF_DEC + DEC_W1 + i * DP + o] * du[o];
                    *scv(a, SC_DH, i, nb0 + j) += v;
                }
                float hb[D], po[D], pi[D], pao[D], pai[D];
                for (int o = 0; o < D; ++o) { hb[o] = h0[(long long)o * a.NB + nb0 + j]; po[o] = 0.f; pi[o] = 0.f; }
                mv_acc<D>(po, Wsh + OFF_OUT + PHI_WB, hb);
                mv_acc<D>(pi, Wsh + OFF_IN + PHI_WB, hb);
                load_vec(pao, Wsh + OFF_OUT + PHI_B1);
                load_vec(pai, Wsh + OFF_IN + PHI_B1);
                mv_acc<D>(pao, Wsh + OFF_OUT + PHI_WA, hb);
                mv_acc<D>(pai, Wsh + OFF_IN + PHI_WA, hb);
                for (int o = 0; o < D; ++o) {
                    *scv(a, SC_PBO, o, nb0 + j) = po[o];
                    *scv(a, SC_PBI, o, nb0 + j) = pi[o];
                    *scv(a, SC_PAO, o, nb0 + j) = pao[o];
                    *scv(a, SC_PAI, o, nb0 + j) = pai[o];
                }
            }
        }
        __syncthreads();
        // (b) messages and Psi recomputed; Psi, second layers backward -> dS_out, dS_in
        for (int pass = 0; pass < n_pass; ++pass) {
            const int j = pass * TR_T + threadIdx.x;
            const bool act = j < nl;
            const bool inner = j < k;
            float h[D], So[D], Si[D], pao[D], pai[D];
            int dout = 0, din = 0;
            for (int o = 0; o < D; ++o) {
                So[o] = 0.f; Si[o] = 0.f;
                h[o] = act ? h0[(long long)o * a.NB + nb0 + j] : 0.f;
                pao[o] = act ? *scv(a, SC_PAO, o, nb0 + j) : 0.f;
                pai[o] = act ? *scv(a, SC_PAI, o, nb0 + j) : 0.f;
            }
            if (act) {
                const float2 xj = xy[j];
                for (int e = gptr[j]; e < gptr[j + 1]; ++e) {
                    const int l = gn[e];
                    const float2 xl = xy[l];
                    const float dx = xl.x - xj.x, dy = xl.y - xj.y, dn = sqrtf(dx * dx + dy * dy);
                    float pbo[D], pbi[D];
                    for (int o = 0; o < D; ++o) { pbo[o] = *scv(a, SC_PBO, o, nb0 + l); pbi[o] = *scv(a, SC_PBI, o, nb0 + l); }
                    if (l < k) { edge_msg(So, pao, pbo, Wsh + OFF_OUT + PHI_WE, dx, dy, dn); ++dout; }
                    if (inner) { edge_msg(Si, pai, pbi, Wsh + OFF_IN + PHI_WE, -dx, -dy, dn); ++din; }
                }
            }
            float fo[D], fi[D];
            for (int o = 0; o < D; ++o) {
                fo[o] = dout * Wsh[OFF_OUT + PHI_B2 + o];
                fi[o] = din * Wsh[OFF_IN + PHI_B2 + o];
            }
            mv_acc<D>(fo, Wsh + OFF_OUT + PHI_W2, So);
            mv_acc<D>(fi, Wsh + OFF_IN + PHI_W2, Si);
            const float cj = act ? a.c[nb0 + j] : 0.f;
            float u[D];
            load_vec(u, Wsh + OFF_PSI + PSI_B1);
            mv_acc<D>(u, Wsh + OFF_PSI + PSI_W1, h);
            float cc[1] = {cj};
            mv_acc<1>(u, Wsh + OFF_PSI + PSI_W1 + D * DP, cc);
            mv_acc<D>(u, Wsh + OFF_PSI + PSI_W1 + (D + 1) * DP, fo);
            mv_acc<D>(u, Wsh + OFF_PSI + PSI_W1 + (2 * D + 1) * DP, fi);
            // Psi backward: d out = alpha dh^{k+1}
            float dout_v[D], du[D];
            for (int o = 0; o < D; ++o) dout_v[o] = act ? a.alpha * *scv(a, SC_DH, o, nb0 + j) : 0.f;
            for (int o = 0; o < D; ++o) gacc(gsh, OFF_PSI + PSI_B2 + o, dout_v[o]);
            for (int i = 0; i < D; ++i) {
                const float ai = relu(u[i]);
                float v = 0.f;
                for (int o = 0; o < D; ++o) {
                    gacc(gsh, OFF_PSI + PSI_W2 + i * DP + o, dout_v[o] * ai);
                    v += Wsh[OFF_PSI + PSI_W2 + i * DP + o] * dout_v[o];
                }
                du[i] = u[i] > 0.f ? v : 0.f;
            }
            for (int o = 0; o < D; ++o) gacc(gsh, OFF_PSI + PSI_B1 + o, du[o]);
            // x = [h, c, phi_out, phi_in]
            float dfo[D], dfi[D];
            for (int i = 0; i < 3 * D + 1; ++i) {
                const float xi = i < D ? h[i] : (i == D ? cj : (i < 2 * D + 1 ? fo[i - D - 1] : fi[i - 2 * D - 1]));
                float v = 0.f;
                for (int o = 0; o < D; ++o) {
                    gacc(gsh, OFF_PSI + PSI_W1 + i * DP + o, du[o] * xi);
                    v += Wsh[OFF_PSI + PSI_W1 + i * DP + o] * du[o];
                }
                if (i < D) {
                    if (act) *scv(a, SC_DH, i, nb0 + j) += v;  // dh^k = dh^{k+1} + dPsi/dh
                } else if (i > D && i < 2 * D + 1) {
                    dfo[i - D - 1] = v;
                } else if (i >= 2 * D + 1) {
                    dfi[i - 2 * D - 1] = v;
                }
            }
            // phi = W2 S + deg b2
            for (int o = 0; o < D; ++o) {
                gacc(gsh, OFF_OUT + PHI_B2 + o, dout * dfo[o]);
                gacc(gsh, OFF_IN + PHI_B2 + o, din * dfi[o]);
            }
            for (int i = 0; i < D; ++i) {
                float vo = 0.f, vi = 0.f;
                for (int o = 0; o < D; ++o) {
                    gacc(gsh, OFF_OUT + PHI_W2 + i * DP + o, dfo[o] * So[i]);
                    gacc(gsh, OFF_IN + PHI_W2 + i * DP + o, dfi[o] * Si[i]);
                    vo += Wsh[OFF_OUT + PHI_W2 + i * DP + o] * dfo[o];
                    vi += Wsh[OFF_IN + PHI_W2 + i * DP + o] * dfi[o];
                }
                if (act) {
                    *scv(a, SC_DSO, i, nb0 + j) = vo;
                    *scv(a, SC_DSI, i, nb0 + j) = vi;
                }
            }
        }
        __syncthreads();
        // (c) edges: dz at the owner; neighbour-projection gradients gathered at their owner
        for (int pass = 0; pass < n_pass; ++pass) {
            const int j = pass * TR_T + threadIdx.x;
            const bool act = j < nl;
            const bool inner = j < k;
            float dpao[D], dpai[D], dpbo[D], dpbi[D], pao[D], pai[D], pbo_j[D], pbi_j[D], dso[D], dsi[D];
            float gWe_o[3][D], gWe_i[3][D];
            for (int o = 0; o < D; ++o) {
                dpao[o] = dpai[o] = dpbo[o] = dpbi[o] = 0.f;
                pao[o] = act ? *scv(a, SC_PAO, o, nb0 + j) : 0.f;
                pai[o] = act ? *scv(a, SC_PAI, o, nb0 + j) : 0.f;
                pbo_j[o] = act ? *scv(a, SC_PBO, o, nb0 + j) : 0.f;
                pbi_j[o] = act ? *scv(a, SC_PBI, o, nb0 + j) : 0.f;
                dso[o] = act ? *scv(a, SC_DSO, o, nb0 + j) : 0.f;
                dsi[o] = act ? *scv(a, SC_DSI, o, nb0 + j) : 0.f;
                for (int f = 0; f < 3; ++f) gWe_o[f][o] = gWe_i[f][o] = 0.f;
            }
            if (act) {
                const float2 xj = xy[j];
                for (int e = gptr[j]; e < gptr[j + 1]; ++e) {
                    const int l = gn[e];
                    const float2 xl = xy[l];
                    const float dx = xl.x - xj.x, dy = xl.y - xj.y, dn = sqrtf(dx * dx + dy * dy);
                    if (l < k) {
                        // own out-message j -> l (feature x_l - x_j)
                        for (int o = 0; o < D; ++o) {
                            float z = pao[o] + *scv(a, SC_PBO, o, nb0 + l) + Wsh[OFF_OUT + PHI_WE + o] * dx +
                                      Wsh[OFF_OUT + PHI_WE + DP + o] * dy + Wsh[OFF_OUT + PHI_WE + 2 * DP + o] * dn;
                            float dz = z > 0.f ? dso[o] : 0.f;
                            dpao[o] += dz;
                            gWe_o[0][o] += dz * dx; gWe_o[1][o] += dz * dy; gWe_o[2][o] += dz * dn;
                        }
                        // l's in-message from j (owner l, feature x_l - x_j): gradient of Pb_in(j)
                        for (int o = 0; o < D; ++o) {
                            float z = *scv(a, SC_PAI, o, nb0 + l) + pbi_j[o] + Wsh[OFF_IN + PHI_WE + o] * dx +
                                      Wsh[OFF_IN + PHI_WE + DP + o] * dy + Wsh[OFF_IN + PHI_WE + 2 * DP + o] * dn;
                            if (z > 0.f) dpbi[o] += *scv(a, SC_DSI, o, nb0 + l);
                        }
                    }
                    if (inner) {
                        // own in-message from l (feature x_j - x_l)
                        for (int o = 0; o < D; ++o) {
                            float z = pai[o] + *scv(a, SC_PBI, o, nb0 + l) - Wsh[OFF_IN + PHI_WE + o] * dx -
                                      Wsh[OFF_IN + PHI_WE + DP + o] * dy + Wsh[OFF_IN + PHI_WE + 2 * DP + o] * dn;
                            float dz = z > 0.f ? dsi[o] : 0.f;
                            dpai[o] += dz;
                            gWe_i[0][o] -= dz * dx; gWe_i[1][o] -= dz * dy; gWe_i[2][o] += dz * dn;
                        }
                        // l's out-message to j (owner l, feature x_j - x_l): gradient of Pb_out(j)
                        for (int o = 0; o < D; ++o) {
                            float z = *scv(a, SC_PAO, o, nb0 + l) + pbo_j[o] - Wsh[OFF_OUT + PHI_WE + o] * dx -
                                      Wsh[OFF_OUT + PHI_WE + DP + o] * dy + Wsh[OFF_OUT + PHI_WE + 2 * DP + o] * dn;
                            if (z > 0.f) dpbo[o] += *scv(a, SC_DSO, o, nb0 + l);
                        }
                    }
                }
            }
            for (int f = 0; f < 3; ++f)
                for (int o = 0; o < D; ++o) {
                    gacc(gsh, OFF_OUT + PHI_WE + f * DP + o, gWe_o[f][o]);
                    gacc(gsh, OFF_IN + PHI_WE + f * DP + o, gWe_i[f][o]);
                }
            for (int o = 0; o < D; ++o) {
                gacc(gsh, OFF_OUT + PHI_B1 + o, dpao[o]);
                gacc(gsh, OFF_IN + PHI_B1 + o, dpai[o]);
            }
            float hb[D];
            for (int i = 0; i < D; ++i) hb[i] = act ? h0[(long long)i * a.NB + nb0 + j] : 0.f;
            for (int i = 0; i < D; ++i) {
                float v = 0.f;
                for (int o = 0; o < D; ++o) {
                    gacc(gsh, OFF_OUT + PHI_WA + i * DP + o, dpao[o] * hb[i]);
                    gacc(gsh, OFF_IN + PHI_WA + i * DP + o, dpai[o] * hb[i]);
                    gacc(gsh, OFF_OUT + PHI_WB + i * DP + o, dpbo[o] * hb[i]);
                    gacc(gsh, OFF_IN + PHI_WB + i * DP + o, dpbi[o] * hb[i]);
                    v += Wsh[OFF_OUT + PHI_WA + i * DP + o] * dpao[o] + Wsh[OFF_IN + PHI_WA + i * DP + o] * dpai[o] +
                         Wsh[OFF_OUT + PHI_WB + i * DP + o] * dpbo[o] + Wsh[OFF_IN + PHI_WB + i * DP + o] * dpbi[o];
                }
                if (act) *scv(a, SC_DH, i, nb0 + j) += v;
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < BLOCK_FLOATS; q += TR_T)
            if (gsh[q] != 0.f) atomicAdd(&a.gpack[(size_t)blk * BLOCK_FLOATS + q], gsh[q]);
    }
}

// ---------------------------------------------------------------- optimiser
// packed index -> flat index (or -1 for padding), one block's pattern
static std::vector<int> packed_to_flat(int d) {
    std::vector<int> map(BLOCK_FLOATS, -1);
    int o0 = 0;
    const int in1 = 2 * D + 3;
    for (int mm = 0; mm < 2; ++mm) {
        const int W1 = o0, b1 = W1 + D * in1, W2 = b1 + D, b2 = W2 + D * D;
        const int base = mm == 0 ? OFF_OUT : OFF_IN;
        for (int oo = 0; oo < D; ++oo) {
            for (int i = 0; i < D; ++i) {
                map[base + PHI_WA + i * DP + oo] = W1 + oo * in1 + i;
                map[base + PHI_WB + i * DP + oo] = W1 + oo * in1 + D + i;
                map[base + PHI_W2 + i * DP + oo] = W2 + oo * D + i;
            }
            for (int i = 0; i < 3; ++i) map[base + PHI_WE + i * DP + oo] = W1 + oo * in1 + 2 * D + i;
            map[base + PHI_B1 + oo] = b1 + oo;
            map[base + PHI_B2 + oo] = b2 + oo;
        }
        o0 = b2 + D;
    }
    const int pW1 = o0, pb1 = pW1 + D * (3 * D + 1), pW2 = pb1 + D, pb2 = pW2 + D * D;
    for (int oo = 0; oo < D; ++oo) {
        for (int i = 0; i < 3 * D + 1; ++i) map[OFF_PSI + PSI_W1 + i * DP + oo] = pW1 + oo * (3 * D + 1) + i;
        for (int i = 0; i < D; ++i) map[OFF_PSI + PSI_W2 + i * DP + oo] = pW2 + oo * D + i;
        map[OFF_PSI + PSI_B1 + oo] = pb1 + oo;
        map[OFF_PSI + PSI_B2 + oo] = pb2 + oo;
    }
    const int dW1 = pb2 + D, db1 = dW1 + D * D, dW2 = db1 + D, db2 = dW2 + D;
    for (int oo = 0; oo < D; ++oo) {
        for (int i = 0; i < D; ++i) map[OFF_DEC + DEC_W1 + i * DP + oo] = dW1 + oo * D + i;
        map[OFF_DEC + DEC_B1 + oo] = db1 + oo;
        map[OFF_DEC + DEC_W2 + oo] = dW2 + oo;
    }
    map[OFF_DEC + DEC_B2] = db2;
    (void)d;
    return map;
}

__global__ void k_tr_unpack_grad(const float *gpack, const int *map, int kbar, int per_block, float *gflat) {
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)kbar * BLOCK_FLOATS) return;
    int blk = (int)(q / BLOCK_FLOATS), r = (int)(q % BLOCK_FLOATS);
    int f = map[r];
    if (f >= 0) gflat[(long long)blk * per_block + f] = gpack[q];
}

__global__ void k_tr_pack(const float *wflat, const int *map, int kbar, int per_block, float *packed) {
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)kbar * BLOCK_FLOATS) return;
    int blk = (int)(q / BLOCK_FLOATS), r = (int)(q % BLOCK_FLOATS);
    int f = map[r];
    packed[q] = f >= 0 ? wflat[(long long)blk * per_block + f] : 0.f;
}

__global__ void k_tr_sumsq(const float *g, long long n, const float *loss, int B, double *out) {
    __shared__ double sh[32];
    double v = 0.0, l = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) v += (double)g[i] * g[i];
    for (int b = threadIdx.x; b < B; b += blockDim.x) l += loss[b];
    v = block_sum(v, sh);
    l = block_sum(l, sh);
    if (threadIdx.x == 0) {
        out[0] = sqrt(v);
        out[1] = l / B;
    }
}

__global__ void k_tr_adam(float *w, const float *g, float *m1, float *m2, long long n, const double *gnorm, float lr,
                          float clip, float bc1, float bc2) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float scale = 1.f;
    if (clip > 0.f && gnorm[0] > clip) scale = (float)(clip / gnorm[0]);
    float gi = g[i] * scale;
    float a = 0.9f * m1[i] + 0.1f * gi;
    float b = 0.999f * m2[i] + 0.001f * gi * gi;
    m1[i] = a;
    m2[i] = b;
    w[i] -= lr * (a / bc1) / (sqrtf(b / bc2) + 1e-8f);
}

// ---------------------------------------------------------------- host driver
struct TrainWork {
    std::vector<void *> bufs;
    ~TrainWork() {
        for (void *b : bufs) cudaFree(b);
    }
    template <class T>
    int32_t get(T **p, size_t n) {
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), (n ? n : 1) * sizeof(T));
        if (e != cudaSuccess) {
            set_error(std::string("training workspace: ") + cudaGetErrorString(e));
            return DDG_OOM;
        }
        bufs.push_back(*p);
        return DDG_OK;
    }
};

// local matrices R_i A R_i^T as per-graph CSR over unknowns (uint16 local columns)
__global__ void k_lm_count(const int *sub_ptr, const int *sub_idx, const int *rowptr, const int *col, const int *mptr,
                           const int *midx, int K, int *cnt) {
    int i = blockIdx.x;
    const int s0 = sub_ptr[i], k = sub_ptr[i + 1] - s0;
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        int f = sub_idx[s0 + t], c = 0;
        for (int e = rowptr[f]; e < rowptr[f + 1]; ++e) {
            int l = col[e];
            for (int q = mptr[l]; q < mptr[l + 1]; ++q) c += midx[q] == i;
        }
        cnt[s0 + i + t] = c;
    }
    if (threadIdx.x == 0) cnt[s0 + i + k] = 0;
}

__global__ void k_lm_fill(const int *sub_ptr, const int *sub_idx, const int *rowptr, const int *col, const double *val,
                          const int *mptr, const int *midx, const int *lm_ptr, uint16_t *lm_col, float *lm_val) {
    int i = blockIdx.x;
    const int s0 = sub_ptr[i], k = sub_ptr[i + 1] - s0;
    const int *S = sub_idx + s0;
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        int f = S[t], o = lm_ptr[s0 + i + t];
        for (int e = rowptr[f]; e < rowptr[f + 1]; ++e) {
            int l = col[e];
            bool in = false;
            for (int q = mptr[l]; q < mptr[l + 1]; ++q) in |= midx[q] == i;
            if (!in) continue;
            int lo = 0, hi = k;
            while (lo < hi) {
                int m = (lo + hi) >> 1;
                if (S[m] < l) lo = m + 1; else hi = m;
            }
            lm_col[o] = (uint16_t)lo;
            lm_val[o] = (float)val[e];
            ++o;
        }
    }
}

struct Trainer {
    ddg_problem *p;
    ddg_model *m;
    TrainWork ws;
    int *lm_ptr = nullptr, *lm_row = nullptr;
    uint16_t *lm_col = nullptr;
    float *lm_val = nullptr;
    int *map = nullptr;
    std::vector<int> nloc, nint;
    int per_block = 0;
    float *gpack = nullptr, *gflat = nullptr, *m1 = nullptr, *m2 = nullptr, *lossb = nullptr;
    double *stats = nullptr;
    // per-batch buffers (sized for the largest batch)
    int cap_B = 0;
    long long cap_NB = 0, cap_NK = 0;
    int *d_graph = nullptr, *d_nbase = nullptr, *d_kbase = nullptr;
    const double **d_res = nullptr;
    float *c = nullptr, *hsave = nullptr, *rhat = nullptr, *ghat = nullptr, *res_k = nullptr, *scr = nullptr;

    int32_t init() {
        cudaStream_t s = p->stream;
        const int K = p->K;
        per_block = 11 * D * D + 15 * D + 1;
        // local matrices
        int *cnt;
        DDG_TRY(ws.get(&cnt, (size_t)p->sum_k + K + 1));
        DDG_TRY(ws.get(&lm_ptr, (size_t)p->sum_k + K + 1));
        k_lm_count<<<K, 256, 0, s>>>(p->sub_ptr, p->sub_idx, p->rowptr, p->col, p->mem_ptr, p->mem_idx, K, cnt);
        DDG_LAUNCH_CHECK();
        int total = 0;
        DDG_TRY(scan_exclusive(p->ctx, cnt, lm_ptr, (int)(p->sum_k + K), &total, s));
        DDG_TRY(ws.get(&lm_col, total));
        DDG_TRY(ws.get(&lm_val, total));
        k_lm_fill<<<K, 256, 0, s>>>(p->sub_ptr, p->sub_idx, p->rowptr, p->col, p->val, p->mem_ptr, p->mem_idx, lm_ptr,
                                    lm_col, lm_val);
        DDG_LAUNCH_CHECK();
        std::vector<int> sp(K + 1), rowstart(K + 1);
        DDG_CU(cudaMemcpyAsync(sp.data(), p->sub_ptr, sizeof(int) * (K + 1), cudaMemcpyDeviceToHost, s));
        std::vector<int> lp(K + 1);
        DDG_CU(cudaMemcpyAsync(lp.data(), p->loc_ptr, sizeof(int) * (K + 1), cudaMemcpyDeviceToHost, s));
        DDG_CU(cudaStreamSynchronize(s));
        nloc.resize(K);
        nint.resize(K);
        for (int i = 0; i < K; ++i) {
            rowstart[i] = sp[i] + i;
            nloc[i] = lp[i + 1] - lp[i];
            nint[i] = sp[i + 1] - sp[i];
        }
        rowstart[K] = sp[K] + K;
        DDG_TRY(ws.get(&lm_row, K + 1));
        DDG_CU(cudaMemcpyAsync(lm_row, rowstart.data(), sizeof(int) * (K + 1), cudaMemcpyHostToDevice, s));
        std::vector<int> hm = packed_to_flat(D);
        DDG_TRY(ws.get(&map, BLOCK_FLOATS));
        DDG_CU(cudaMemcpyAsync(map, hm.data(), sizeof(int) * BLOCK_FLOATS, cudaMemcpyHostToDevice, s));
        const long long nw = (long long)m->kbar * per_block;
        DDG_TRY(ws.get(&gpack, (size_t)m->kbar * BLOCK_FLOATS));
        DDG_TRY(ws.get(&gflat, nw));
        DDG_TRY(ws.get(&stats, 4));
        if (!m->adam_m) {
            DDG_TRY(dalloc(m->ctx, m->allocs, &m->adam_m, nw));
            DDG_TRY(dalloc(m->ctx, m->allocs, &m->adam_v, nw));
            DDG_CU(cudaMemsetAsync(m->adam_m, 0, sizeof(float) * nw, s));
            DDG_CU(cudaMemsetAsync(m->adam_v, 0, sizeof(float) * nw, s));
            m->adam_t = 0;
        }
        m1 = m->adam_m;
        m2 = m->adam_v;
        return DDG_OK;
    }

    int32_t ensure(int B, long long NB, long long NK) {
        if (B <= cap_B && NB <= cap_NB && NK <= cap_NK) return DDG_OK;
        cap_B = std::max(B, cap_B);
        cap_NB = std::max(NB, cap_NB);
        cap_NK = std::max(NK, cap_NK);
        const int kb = m->kbar;
        DDG_TRY(ws.get(&d_graph, cap_B));
        DDG_TRY(ws.get(&d_nbase, cap_B + 1));
        DDG_TRY(ws.get(&d_kbase, cap_B + 1));
        DDG_TRY(ws.get(&d_res, cap_B));
        DDG_TRY(ws.get(&lossb, cap_B));
        DDG_TRY(ws.get(&c, cap_NB));
        DDG_TRY(ws.get(&hsave, (size_t)(kb + 1) * D * cap_NB));
        DDG_TRY(ws.get(&rhat, (size_t)kb * cap_NK));
        DDG_TRY(ws.get(&ghat, (size_t)kb * cap_NK));
        DDG_TRY(ws.get(&res_k, cap_NK));
        DDG_TRY(ws.get(&scr, (size_t)8 * D * cap_NB));
        return DDG_OK;
    }

    // loss (mean over the batch) and gradient in gflat for samples (graph, residual pointer)
    int32_t loss_grad(const std::vector<int> &graphs, const std::vector<const double *> &res, double *loss_out) {
        cudaStream_t s = p->stream;
        const int B = (int)graphs.size();
        std::vector<int> nb(B + 1, 0), kb(B + 1, 0);
        for (int b = 0; b < B; ++b) {
            nb[b + 1] = nb[b] + nloc[graphs[b]];
            kb[b + 1] = kb[b] + nint[graphs[b]];
        }
        DDG_TRY(ensure(B, nb[B], kb[B]));
        DDG_CU(cudaMemcpyAsync(d_graph, graphs.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
        DDG_CU(cudaMemcpyAsync(d_nbase, nb.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice, s));
        DDG_CU(cudaMemcpyAsync(d_kbase, kb.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice, s));
        DDG_CU(cudaMemcpyAsync(d_res, res.data(), sizeof(double *) * B, cudaMemcpyHostToDevice, s));
        DDG_CU(cudaMemsetAsync(gpack, 0, sizeof(float) * m->kbar * BLOCK_FLOATS, s));
        TrainArgs a{};
        a.W = m->packed;
        a.kbar = m->kbar;
        a.alpha = m->alpha;
        a.B = B;
        a.graph = d_graph;
        a.res = d_res;
        a.nbase = d_nbase;
        a.kbase = d_kbase;
        a.NB = cap_NB;
        a.NK = cap_NK;
        a.loc_ptr = p->loc_ptr;
        a.loc_nint = p->loc_nint;
        a.nbr_ptr = p->nbr_ptr;
        a.nbr_off = p->nbr_off;
        a.sub_ptr = p->sub_ptr;
        a.sub_idx = p->sub_idx;
        a.nbr = p->nbr;
        a.loc_xy = p->loc_xy;
        a.lm_ptr = lm_ptr;
        a.lm_row = lm_row;
        a.lm_col = lm_col;
        a.lm_val = lm_val;
        a.c = c;
        a.hsave = hsave;
        a.rhat = rhat;
        a.ghat = ghat;
        a.res_k = res_k;
        a.scr = scr;
        a.gpack = gpack;
        a.loss = lossb;
        k_tr_fwd<<<B, TR_T, 0, s>>>(a);
        DDG_LAUNCH_CHECK();
        k_tr_bwd<<<B, TR_T, 0, s>>>(a);
        DDG_LAUNCH_CHECK();
        const long long nw = (long long)m->kbar * per_block;
        DDG_CU(cudaMemsetAsync(gflat, 0, sizeof(float) * nw, s));
        k_tr_unpack_grad<<<cdiv((long long)m->kbar * BLOCK_FLOATS, 256), 256, 0, s>>>(gpack, map, m->kbar, per_block,
                                                                                     gflat);
        DDG_LAUNCH_CHECK();
        k_tr_sumsq<<<1, 256, 0, s>>>(gflat, nw, lossb, B, stats);
        DDG_LAUNCH_CHECK();
        if (loss_out) {
            double st[2];
            DDG_CU(cudaMemcpyAsync(st, stats, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
            DDG_CU(cudaStreamSynchronize(s));
            *loss_out = st[1];
        }
        return DDG_OK;
    }

    int32_t adam_step(int t, float lr, float clip) {
        cudaStream_t s = p->stream;
        const long long nw = (long long)m->kbar * per_block;
        float bc1 = 1.f - std::pow(0.9f, (float)t), bc2 = 1.f - std::pow(0.999f, (float)t);
        k_tr_adam<<<cdiv(nw, 256), 256, 0, s>>>(m->w, gflat, m1, m2, nw, stats, lr, clip, bc1, bc2);
        k_tr_pack<<<cdiv((long long)m->kbar * BLOCK_FLOATS, 256), 256, 0, s>>>(m->w, map, m->kbar, per_block,
                                                                             m->packed);
        DDG_LAUNCHES(2);
        return DDG_OK;
    }
};

static uint64_t sm_next(uint64_t &state) {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int32_t train_local_model(ddg_problem *p, ddg_model *m, const ddg_train_opts *o, ddg_train_report *rep) {
    cudaStream_t s = p->stream;
    cudaEvent_t e0, e1;
    DDG_CU(cudaEventCreate(&e0));
    DDG_CU(cudaEventCreate(&e1));
    DDG_CU(cudaEventRecord(e0, s));
    // harvest: residuals of DDM-LU preconditioned CG iterations
    DDG_TRY(ddg_setup_precond(p, DDG_DDM_LU, nullptr, DDG_COARSE));
    Trainer tr;
    tr.p = p;
    tr.m = m;
    double *bank = nullptr;
    DDG_TRY(tr.ws.get(&bank, (size_t)o->harvest_iters * p->nf));
    int stored = 0;
    DDG_TRY(fcg_solve_record(p, o->harvest_iters, bank, &stored));
    DDG_TRY(tr.init());
    const int K = p->K;
    const int n_samples = K * stored;
    uint64_t rng = o->seed;
    double lr = o->lr, best = 1e300;
    int since_best = 0;
    double first = -1.0, last = 0.0, window = 0.0;
    int win_n = 0;
    for (int step = 1; step <= o->steps; ++step) {
        std::vector<int> graphs(o->batch);
        std::vector<const double *> res(o->batch);
        for (int b = 0; b < o->batch; ++b) {
            int q = (int)(sm_next(rng) % (uint64_t)n_samples);
            graphs[b] = q % K;
            res[b] = bank + (size_t)(q / K) * p->nf;
        }
        double loss = 0.0;
        DDG_TRY(tr.loss_grad(graphs, res, &loss));
        DDG_TRY(tr.adam_step((int)(++m->adam_t), (float)lr, o->clip));
        if (first < 0.0) first = loss;
        last = loss;
        window += loss;
        ++win_n;
        if (win_n == 50) {  // plateau schedule on 50-step windows (factor 0.1, patience 8 windows)
            double mean = window / win_n;
            if (mean < best * 0.999) {
                best = mean;
                since_best = 0;
            } else if (++since_best >= 8) {
                lr *= 0.1;
                since_best = 0;
            }
            window = 0.0;
            win_n = 0;
        }
    }
    DDG_CU(cudaEventRecord(e1, s));
    DDG_CU(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    DDG_TRY(model_host_layouts(m));
    if (rep) {
        rep->samples = n_samples;
        rep->steps = o->steps;
        rep->loss_first = first;
        rep->loss_last = last;
        rep->ms = ms;
        rep->lr_final = lr;
    }
    return DDG_OK;
}

int32_t train_loss_grad(ddg_problem *p, ddg_model *m, const double *r_dev, const int *graphs_host, int nb,
                        double *loss, float *grad_host) {
    Trainer tr;
    tr.p = p;
    tr.m = m;
    DDG_TRY(tr.init());
    std::vector<int> graphs(graphs_host, graphs_host + nb);
    std::vector<const double *> res(nb, r_dev);
    DDG_TRY(tr.loss_grad(graphs, res, loss));
    if (grad_host) {
        DDG_CU(cudaMemcpy(grad_host, tr.gflat, sizeof(float) * m->n_w, cudaMemcpyDeviceToHost));
    }
    return DDG_OK;
}

}  // namespace ddg
