// Adjoint (vector-Jacobian product) of the cluster pair forces.
//
// The paper has no adjoint; this kernel differentiates the pair kernel of
// Sec. V.A.  For L = <gF, F> + gE * (E_LJ + E_C) it recomputes every pair of
// the inner list (nothing is stored by the forward pass) and accumulates, per
// pair with d = x_i - x_j (image), w = gF_i - gF_j, u = d . w:
//   dL/dx_i += phi w + (phi'/r) u d - gE phi d          (minus that on x_j)
//   dL/dq_i += q_j (psi_C u + gE v_C)                   (and q_i (...) on q_j)
//   dL/dC12[a][b] += 12 r^-14 u + gE (r^-12 - rc^-12)
//   dL/dC6[a][b]  += -6 r^-8 u - gE (r^-6 - rc^-6)
// with phi = -(1/r) dV/dr, phi_C = qi qj psi_C, V_C = qi qj v_C.  The loop
// structure is the force kernel's: one warp per work item, lanes (ti, tj)
// over the 8x8 cluster pair, i-gradients in registers, j-gradients reduced
// over the ti lanes per j-entry.  Parameter gradients are accumulated in shared
// memory (FP32, one item), then added to an FP64 table; the table is symmetrised
// at the end so that a type pair a != b puts half of its gradient in [a][b] and
// half in [b][a] (the pair parameter is (C[a][b] + C[b][a]) / 2).  With up to 8
// atom types every lane owns a column of the accumulators ([type pair][33],
// conflict-free) and the warp folds the columns once per item; with more types
// the lanes add into one table per warp with shared-memory atomics.  (A few type
// pairs shared by all 32 lanes serialise such atomics: on the 6-type 24k water box
// they took two thirds of the kernel.)
#include "nb_pair.cuh"

using namespace nbk;

namespace {

constexpr int kVW = 4;
constexpr int kVjpMaxT = 16;     // shared-memory parameter accumulators (T*T per warp)
constexpr int kVjpPrivMaxT = 8;  // per-lane accumulator columns up to this many types
constexpr int kColStride = 33;   // column stride of the per-lane accumulators (bank-conflict free)

struct VjpView {
    SysView s;
    const float4 *gf;  // sorted gF (xyz)
    float4 *gx;        // sorted dL/dx accumulators
    float *gq;         // sorted dL/dq accumulators
    double *gpar;      // [2*T*T] unsymmetrised dL/dC6, dL/dC12
    float gE;
    float two_beta_sqrtpi;  // 2 beta / sqrt(pi)
};

template <int COUL, bool PRIV>
__global__ void __launch_bounds__(kVW * 32) k_vjp(VjpView v) {
    __shared__ float4 s_xi[kVW][NB_SCA];
    __shared__ float4 s_gi[kVW][NB_SCA];
    __shared__ int s_ti[kVW][NB_SCA];
    __shared__ float4 s_lje[kVjpMaxT * kVjpMaxT];
    extern __shared__ float s_par[];  // PRIV: [kVW][2][T*T][33]; else [kVW][2][T*T]
    const SysView &sv = v.s;
    const int T = sv.T, TT = T * T;
    for (int t = threadIdx.x; t < TT; t += blockDim.x) s_lje[t] = sv.lje[t];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *const p6 = s_par + (size_t)wib * 2 * TT * (PRIV ? kColStride : 1);
    float *const p12 = p6 + TT * (PRIV ? kColStride : 1);
    if (PRIV) {
        for (int t = 0; t < TT; t++) {
            p6[t * kColStride + lane] = 0.f;
            p12[t * kColStride + lane] = 0.f;
        }
    } else {
        for (int t = lane; t < TT; t += 32) {
            p6[t] = 0.f;
            p12[t] = 0.f;
        }
    }
    __syncthreads();
    const int w = blockIdx.x * kVW + wib;
    if (w >= sv.n_items) return;
    const int nj = sv.inner_len[w];
    if (nj == 0) return;
    const int4 it = sv.items[w];
    const int si = it.x, j0 = it.z;
    const ShiftSplit sh = make_shift(it.y, sv.box_hi, sv.box_lo);
    for (int h = 0; h < 2; h++) {
        const int at = lane + 32 * h;
        s_xi[wib][at] = shift_i(sv.xq[si * NB_SCA + at], sh);
        s_gi[wib][at] = v.gf[si * NB_SCA + at];
        s_ti[wib][at] = sv.type[si * NB_SCA + at];
    }
    __syncwarp();
    const int ti = lane & 7, tj = lane >> 3;
    const unsigned full = 0xffffffffu;
    const float f = sv.coul_f, gE = v.gE;
    float gix[NB_SCL], giy[NB_SCL], giz[NB_SCL], giq[NB_SCL];
#pragma unroll
    for (int k = 0; k < NB_SCL; k++) gix[k] = giy[k] = giz[k] = giq[k] = 0.f;

    for (int e = 0; e < nj; e++) {
        const int2 ent = sv.cj[j0 + e];
        const int cj = inner_cj(ent), mg = entry_group(ent), lo = inner_lo(ent), hi = inner_hi(ent);
        const int im = lo | hi;
        float4 xj[2], gj[2];
        int tjt[2];
        float ajx[2] = {0.f, 0.f}, ajy[2] = {0.f, 0.f}, ajz[2] = {0.f, 0.f}, ajq[2] = {0.f, 0.f};
        for (int h = 0; h < 2; h++) {
            xj[h] = shift_j(sv.xq[cj * NB_CL + tj + 4 * h], sh);
            gj[h] = v.gf[cj * NB_CL + tj + 4 * h];
            tjt[h] = sv.type[cj * NB_CL + tj + 4 * h];
        }
#pragma unroll
        for (int k = 0; k < NB_SCL; k++) {
            if (!(im & (1 << k))) continue;
            const unsigned long long m = mg ? sv.masks[(size_t)(mg - 1) * 8 + k] : ~0ull;
            const float4 xi = s_xi[wib][k * NB_CL + ti];
            const float4 gi = s_gi[wib][k * NB_CL + ti];
            const int ta = s_ti[wib][k * NB_CL + ti];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                if (!(((h ? hi : lo) >> k) & 1)) continue;  // j-half pruned away (warp-uniform)
                const bool bit = (m >> (ti * 8 + tj + 4 * h)) & 1ull;
                const float dx = xi.x - xj[h].x, dy = xi.y - xj[h].y, dz = xi.z - xj[h].z;
                float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const bool in = bit && (r2 < sv.rc2);
                r2 = in ? r2 : sv.rc2;
                float rinv = rsqrtf(r2);
                rinv = rsqrt_refine(r2, rinv);
                const float rinv2 = rinv * rinv;
                const float rinv6 = rinv2 * rinv2 * rinv2;
                const float rinv8 = rinv6 * rinv2;
                const float rinv12 = rinv6 * rinv6;
                const float rinv14 = rinv12 * rinv2;
                const float4 le = s_lje[ta * T + tjt[h]];  // (C6, C12, shift, -)
                const float phi_lj = fmaf(12.f * le.y, rinv14, -6.f * le.x * rinv8);
                const float dphi_lj = fmaf(-168.f * le.y, rinv14 * rinv2, 48.f * le.x * rinv8 * rinv2);
                const float qq = xi.w * xj[h].w;
                float psi = 0.f, dpsi = 0.f, vcu = 0.f;
                if (COUL == NB_COULOMB_RF) {
                    psi = f * fmaf(rinv, rinv2, -2.f * sv.k_rf);
                    dpsi = -3.f * f * rinv2 * rinv2 * rinv;
                    vcu = f * ((rinv - sv.c_rf) + fmaf(sv.k_rf, r2, -sv.c_rf_lo));
                } else if (COUL == NB_COULOMB_EWALD) {
                    const float r = r2 * rinv;
                    const float z = sv.ew_beta * r;
                    const float ez = __expf(-z * z);
                    const float t = z * (1.0f / NB_EW_ZMAX);
                    float xp = fmaf(NB_EW_XP4, t, NB_EW_XP3);
                    xp = fmaf(xp, t, NB_EW_XP2);
                    xp = fmaf(xp, t, NB_EW_XP1);
                    xp = fmaf(xp, t, NB_EW_XP0);
                    float xq = fmaf(NB_EW_XQ4, t, NB_EW_XQ3);
                    xq = fmaf(xq, t, NB_EW_XQ2);
                    xq = fmaf(xq, t, NB_EW_XQ1);
                    xq = fmaf(xq, t, 1.0f);
                    const float ec = ez * __fdividef(xp, xq);
                    const float ex = v.two_beta_sqrtpi * ez;
                    psi = f * fmaf(ec, rinv, ex) * rinv2;
                    dpsi = f * (-3.f * ec * rinv2 * rinv2 * rinv -
                                ex * fmaf(3.f, rinv2 * rinv2, 2.f * sv.ew_beta * sv.ew_beta * rinv2));
                    vcu = f * fmaf(ec, rinv, -sv.ew_shift);
                }
                float phi = fmaf(qq, psi, phi_lj);
                float dphir = fmaf(qq, dpsi, dphi_lj);
                const float wx = gi.x - gj[h].x, wy = gi.y - gj[h].y, wz = gi.z - gj[h].z;
                const float u = fmaf(dz, wz, fmaf(dy, wy, dx * wx));
                const float cu = fmaf(dphir, u, -gE * phi);
                float gxv = fmaf(phi, wx, cu * dx), gyv = fmaf(phi, wy, cu * dy), gzv = fmaf(phi, wz, cu * dz);
                float gqc = fmaf(psi, u, gE * vcu);
                float g12 = fmaf(12.f * rinv14, u, gE * (rinv12 - sv.rc12inv));
                float g6 = fmaf(-6.f * rinv8, u, -gE * (rinv6 - sv.rc6inv));
                if (!in) gxv = gyv = gzv = gqc = g12 = g6 = 0.f;
                gix[k] += gxv;
                giy[k] += gyv;
                giz[k] += gzv;
                giq[k] += xj[h].w * gqc;
                ajx[h] -= gxv;
                ajy[h] -= gyv;
                ajz[h] -= gzv;
                ajq[h] += xi.w * gqc;
                if (PRIV) {  // g6, g12 are zero for pairs outside rc
                    p6[(ta * T + tjt[h]) * kColStride + lane] += g6;
                    p12[(ta * T + tjt[h]) * kColStride + lane] += g12;
                } else if (in) {
                    atomicAdd(&p6[ta * T + tjt[h]], g6);
                    atomicAdd(&p12[ta * T + tjt[h]], g12);
                }
            }
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            for (int h = 0; h < 2; h++) {
                ajx[h] += __shfl_xor_sync(full, ajx[h], o);
                ajy[h] += __shfl_xor_sync(full, ajy[h], o);
                ajz[h] += __shfl_xor_sync(full, ajz[h], o);
                ajq[h] += __shfl_xor_sync(full, ajq[h], o);
            }
        }
        if (ti == 0) {
            for (int h = 0; h < 2; h++) {
                atomicAdd(&v.gx[cj * NB_CL + tj + 4 * h], make_float4(ajx[h], ajy[h], ajz[h], 0.f));
                atomicAdd(&v.gq[cj * NB_CL + tj + 4 * h], ajq[h]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NB_SCL; k++) {
        for (int o = 8; o < 32; o <<= 1) {
            gix[k] += __shfl_xor_sync(full, gix[k], o);
            giy[k] += __shfl_xor_sync(full, giy[k], o);
            giz[k] += __shfl_xor_sync(full, giz[k], o);
            giq[k] += __shfl_xor_sync(full, giq[k], o);
        }
    }
    if (tj == 0) {
        for (int k = 0; k < NB_SCL; k++) {
            atomicAdd(&v.gx[si * NB_SCA + k * NB_CL + ti], make_float4(gix[k], giy[k], giz[k], 0.f));
            atomicAdd(&v.gq[si * NB_SCA + k * NB_CL + ti], giq[k]);
        }
    }
    __syncwarp();
    for (int t = lane; t < TT; t += 32) {
        float a = 0.f, b = 0.f;
        if (PRIV) {  // lane t folds row t over the 32 lane columns (banks (t + l) mod 32)
            for (int l = 0; l < 32; l++) {
                a += p6[t * kColStride + l];
                b += p12[t * kColStride + l];
            }
        } else {
            a = p6[t];
            b = p12[t];
        }
        if (a != 0.f) atomicAdd(&v.gpar[t], (double)a);
        if (b != 0.f) atomicAdd(&v.gpar[TT + t], (double)b);
    }
}

__global__ void k_vjp_gather(int nslots, const int *__restrict__ perm, const float *__restrict__ x,
                             const int *__restrict__ img, const float *__restrict__ q_s,
                             const float *__restrict__ gF, double Lx, double Ly, double Lz, float4 *__restrict__ xq,
                             float4 *__restrict__ gf, float4 *__restrict__ gx, float *__restrict__ gq, double *gpar,
                             int n_par, int *err) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n_par) gpar[s] = 0.0;
    if (s >= nslots) return;
    gx[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    gq[s] = 0.f;
    const int i = perm[s];
    if (i < 0) {
        gf[s] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    float p[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    int n[3];
    img_unpack(img[i], n[0], n[1], n[2]);
    const double L[3] = {Lx, Ly, Lz};
    bool bad = false;
    for (int k = 0; k < 3; k++) {
        if (!isfinite(p[k])) {
            bad = true;
            p[k] = 0.f;
        } else if (n[k] != 0) {
            p[k] = (float)((double)p[k] - (double)n[k] * L[k]);
        }
    }
    float g[3] = {gF[3 * i], gF[3 * i + 1], gF[3 * i + 2]};
    for (int k = 0; k < 3; k++) {
        if (!isfinite(g[k])) {
            bad = true;
            g[k] = 0.f;
        }
    }
    if (bad) record_error(err, NB_ERR_NONFINITE);
    xq[s] = make_float4(p[0], p[1], p[2], q_s[s]);
    gf[s] = make_float4(g[0], g[1], g[2], 0.f);
}

__global__ void k_vjp_finish(int n, const int *__restrict__ inv, const float4 *__restrict__ gxs,
                             const float *__restrict__ gqs, float *__restrict__ gx, float *__restrict__ gq, int T,
                             const double *__restrict__ gpar, double *gc6, double *gc12) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int s = inv[i];
        const float4 v = gxs[s];
        gx[3 * i] = v.x;
        gx[3 * i + 1] = v.y;
        gx[3 * i + 2] = v.z;
        gq[i] = gqs[s];
    }
    if (i < T * T) {
        const int a = i / T, b = i % T;
        const int TT = T * T;
        gc6[i] = 0.5 * (gpar[a * T + b] + gpar[b * T + a]);
        gc12[i] = 0.5 * (gpar[TT + a * T + b] + gpar[TT + b * T + a]);
    }
}

template <int COUL, bool PRIV>
void launch_vjp(const VjpView &v, int nb, size_t smem, cudaStream_t st) {
    // the default limit of 48 KB covers static and dynamic shared memory together
    if (smem > 16 * 1024) cudaFuncSetAttribute(k_vjp<COUL, PRIV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_vjp<COUL, PRIV><<<nb, kVW * 32, smem, st>>>(v);
}

}  // namespace

nb_status nb_launch_vjp(nb_ctx *c, const float *x, const float *gF, double gE, float *gx, float *gq, double *gc6,
                        double *gc12, cudaStream_t st) {
    if (c->T > kVjpMaxT) return NB_ERR_INVALID_ARG;
    const int ns = c->S_host * NB_SCA;
    const int npar = 2 * c->T * c->T;
    const int nthr = ns > npar ? ns : npar;
    k_vjp_gather<<<(nthr + 255) / 256, 256, 0, st>>>(ns, c->perm, x, c->img, c->q_s, gF, c->box[0], c->box[1],
                                                      c->box[2], c->xq, c->gfs, c->gxs, c->gqs, c->gpar, npar,
                                                      c->err);
    VjpView v;
    v.s = nb_make_view(c, c->fs, nullptr, nullptr);
    v.gf = c->gfs;
    v.gx = c->gxs;
    v.gq = c->gqs;
    v.gpar = c->gpar;
    v.gE = (float)gE;
    v.two_beta_sqrtpi = (float)(2.0 * c->beta / sqrt(M_PI));
    c->n_launches += 2;
    if (v.s.n_items > 0) {
        NbTraceScope tr(c, NB_TRACE_VJP, st);
        c->n_launches++;
        const int nb = (v.s.n_items + kVW - 1) / kVW;
        const int TT = c->T * c->T;
        if (c->T <= kVjpPrivMaxT) {
            const size_t smem = sizeof(float) * kVW * 2 * TT * kColStride;
            if (c->coulomb == NB_COULOMB_RF)
                launch_vjp<NB_COULOMB_RF, true>(v, nb, smem, st);
            else if (c->coulomb == NB_COULOMB_EWALD)
                launch_vjp<NB_COULOMB_EWALD, true>(v, nb, smem, st);
            else
                launch_vjp<NB_COULOMB_NONE, true>(v, nb, smem, st);
        } else {
            const size_t smem = sizeof(float) * kVW * 2 * TT;
            if (c->coulomb == NB_COULOMB_RF)
                launch_vjp<NB_COULOMB_RF, false>(v, nb, smem, st);
            else if (c->coulomb == NB_COULOMB_EWALD)
                launch_vjp<NB_COULOMB_EWALD, false>(v, nb, smem, st);
            else
                launch_vjp<NB_COULOMB_NONE, false>(v, nb, smem, st);
        }
    }
    const int nf = c->N > c->T * c->T ? c->N : c->T * c->T;
    k_vjp_finish<<<(nf + 255) / 256, 256, 0, st>>>(c->N, c->inv, c->gxs, c->gqs, gx, gq, c->T, c->gpar, gc6, gc12);
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}
