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
// memory per unordered type pair (FP32, one item), then added to an FP64 table;
// the table is symmetrised at the end so that a type pair a != b puts half of its
// gradient in [a][b] and half in [b][a] (the pair parameter is (C[a][b] +
// C[b][a]) / 2).  With up to 8 atom types every lane owns a column of the
// accumulators ([unordered type pair][33], conflict-free; T (T + 1) / 2 rows
// instead of T^2 keep the shared memory of 4 warps low enough for 4 resident
// blocks per SM up to 6 types) and the warp folds the columns once per item; with more types
// the lanes add into one table per warp with shared-memory atomics.  (A few type
// pairs shared by all 32 lanes serialise such atomics: on the 6-type 24k water box
// they took two thirds of the kernel.)
#include <algorithm>

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
    float gE;          // the energy's weight, or
    const double *gE_dev;  // read from device memory when not null (no host synchronisation)
    float two_beta_sqrtpi;  // 2 beta / sqrt(pi)
};

// Gradient terms of one pair (formulas in the header comment): g, the dL/dx
// contribution on i (its negative goes to j); gqc, the charge factor
// (dL/dq_i += q_j gqc, dL/dq_j += q_i gqc); g6 and g12, the parameter terms.
// All are zero for a pair that is excluded or outside rc; the result says
// whether the pair counts.
template <int COUL>
__device__ __forceinline__ bool vjp_pair(const VjpView &v, const float4 *__restrict__ lje, float3 d, float3 wv,
                                         float qi, float qj, int tpair, bool bit, float gE, float3 &g, float &gqc,
                                         float &g6, float &g12, int &tsym) {
    const SysView &sv = v.s;
    const float f = sv.coul_f;
    float r2 = fmaf(d.z, d.z, fmaf(d.y, d.y, d.x * d.x));
    const bool in = bit && (r2 < sv.rc2);
    r2 = in ? r2 : sv.rc2;
    float rinv = rsq_approx(r2);
    rinv = rsqrt_refine(r2, rinv);
    const float rinv2 = rinv * rinv;
    const float rinv6 = rinv2 * rinv2 * rinv2;
    const float rinv8 = rinv6 * rinv2;
    const float rinv12 = rinv6 * rinv6;
    const float rinv14 = rinv12 * rinv2;
    const float4 le = lje[tpair];  // (C6, C12, shift, unordered type-pair index)
    tsym = __float_as_int(le.w);
    const float phi_lj = fmaf(12.f * le.y, rinv14, -6.f * le.x * rinv8);
    const float dphi_lj = fmaf(-168.f * le.y, rinv14 * rinv2, 48.f * le.x * rinv8 * rinv2);
    const float qq = qi * qj;
    float psi = 0.f, dpsi = 0.f, vcu = 0.f;
    if (COUL == NB_COULOMB_RF) {
        psi = f * fmaf(rinv, rinv2, -2.f * sv.k_rf);
        dpsi = -3.f * f * rinv2 * rinv2 * rinv;
        vcu = f * ((rinv - sv.c_rf) + fmaf(sv.k_rf, r2, -sv.c_rf_lo));
    } else if (COUL == NB_COULOMB_EWALD) {
        const float r = r2 * rinv;
        const float z = sv.ew_beta * r;
        const float ez = ex2_approx(-z * z * 1.44269504f);  // exp(-z^2)
        const float ec = ez * ew_x(z * (1.0f / NB_EW_ZMAX));
        const float ex = v.two_beta_sqrtpi * ez;
        psi = f * fmaf(ec, rinv, ex) * rinv2;
        dpsi = f * (-3.f * ec * rinv2 * rinv2 * rinv - ex * fmaf(3.f, rinv2 * rinv2, 2.f * sv.ew_beta * sv.ew_beta * rinv2));
        vcu = f * fmaf(ec, rinv, -sv.ew_shift);
    }
    const float phi = fmaf(qq, psi, phi_lj);
    const float dphir = fmaf(qq, dpsi, dphi_lj);
    const float u = fmaf(d.z, wv.z, fmaf(d.y, wv.y, d.x * wv.x));
    const float cu = fmaf(dphir, u, -gE * phi);
    g = make_float3(fmaf(phi, wv.x, cu * d.x), fmaf(phi, wv.y, cu * d.y), fmaf(phi, wv.z, cu * d.z));
    gqc = fmaf(psi, u, gE * vcu);
    g12 = fmaf(12.f * rinv14, u, gE * (rinv12 - sv.rc12inv));
    g6 = fmaf(-6.f * rinv8, u, -gE * (rinv6 - sv.rc6inv));
    if (!in) {
        g = make_float3(0.f, 0.f, 0.f);
        gqc = g6 = g12 = 0.f;
    }
    return in;
}

// Parameter terms of one pair into this lane's column (PRIV) or the warp's table.
template <bool PRIV>
__device__ __forceinline__ void add_par(float *p6, float *p12, int tp, int lane, bool in, float g6, float g12) {
    if (PRIV) {  // zero for pairs that do not count
        p6[tp * kColStride + lane] += g6;
        p12[tp * kColStride + lane] += g12;
    } else if (in) {
        atomicAdd(&p6[tp], g6);
        atomicAdd(&p12[tp], g12);
    }
}

// One work item (the force kernel's loop structure): i-atom positions, incoming
// force gradients and types staged in shared memory, i-gradient accumulators in
// shared memory ([cluster][x, y, z, q][lane]), j-gradients in registers reduced
// over the 8 ti lanes per entry; the i-cluster loop walks the set bits of the
// half masks, two pairs per lane where both j-halves are kept.
template <int COUL, bool PRIV>
__device__ __forceinline__ void vjp_item(const VjpView &v, int w, int nj, float4 *s_xi, float4 *s_gi, int *s_ti,
                                         float *s_ga, const float4 *lje, float *p6, float *p12, int T, float gE) {
    const SysView &sv = v.s;
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const int4 it = sv.items[w];
    const int si = it.x, j0 = it.z;
    const ShiftSplit sh = make_shift(it.y, sv.box_hi, sv.box_lo);
    for (int h = 0; h < 2; h++) {
        const int at = lane + 32 * h;
        s_xi[at] = shift_i(sv.xq[si * NB_SCA + at], sh);
        s_gi[at] = v.gf[si * NB_SCA + at];
        s_ti[at] = sv.type[si * NB_SCA + at];
    }
#pragma unroll
    for (int k = 0; k < 4 * NB_SCL; k++) s_ga[k * 32 + lane] = 0.f;
    __syncwarp();
    const int ti = lane & 7, tj = lane >> 3;
    for (int e = 0; e < nj; e++) {
        const int2 ent = sv.cj[j0 + e];
        const int cj = inner_cj(ent), mg = entry_group(ent), lo = inner_lo(ent), hi = inner_hi(ent);
        float4 xj0 = sv.xq[cj * NB_CL + tj], xj1 = sv.xq[cj * NB_CL + tj + 4];
        if (sh.jshift) {
            xj0 = shift_j(xj0, sh);
            xj1 = shift_j(xj1, sh);
        }
        const float4 gj0 = v.gf[cj * NB_CL + tj], gj1 = v.gf[cj * NB_CL + tj + 4];
        const int tb0 = sv.type[cj * NB_CL + tj], tb1 = sv.type[cj * NB_CL + tj + 4];
        // exclusion bits of the lane's two pairs for every i-cluster k (bits 2k, 2k + 1)
        const unsigned mw = mg ? (unsigned)sv.mask_lanes[(size_t)(mg - 1) * 32 + lane] : 0xffffu;
        float a0x = 0.f, a0y = 0.f, a0z = 0.f, a0q = 0.f, a1x = 0.f, a1y = 0.f, a1z = 0.f, a1q = 0.f;
        int both = lo & hi;
#pragma unroll 1
        while (both) {
            const int k = __ffs(both) - 1;
            both &= both - 1;
            const bool b0 = (mw >> (2 * k)) & 1u, b1 = (mw >> (2 * k + 1)) & 1u;
            const float4 xi = s_xi[k * NB_CL + ti];
            const float4 gi = s_gi[k * NB_CL + ti];
            const int ta = s_ti[k * NB_CL + ti];
            float3 g0, g1;
            float q0, q1, c60, c61, c120, c121;
            int u0, u1;
            const bool in0 = vjp_pair<COUL>(v, lje, make_float3(xi.x - xj0.x, xi.y - xj0.y, xi.z - xj0.z),
                                            make_float3(gi.x - gj0.x, gi.y - gj0.y, gi.z - gj0.z), xi.w, xj0.w,
                                            ta * T + tb0, b0, gE, g0, q0, c60, c120, u0);
            const bool in1 = vjp_pair<COUL>(v, lje, make_float3(xi.x - xj1.x, xi.y - xj1.y, xi.z - xj1.z),
                                            make_float3(gi.x - gj1.x, gi.y - gj1.y, gi.z - gj1.z), xi.w, xj1.w,
                                            ta * T + tb1, b1, gE, g1, q1, c61, c121, u1);
            float *ga = s_ga + k * 128 + lane;
            ga[0] += g0.x + g1.x;
            ga[32] += g0.y + g1.y;
            ga[64] += g0.z + g1.z;
            ga[96] += fmaf(xj0.w, q0, xj1.w * q1);
            a0x -= g0.x;
            a0y -= g0.y;
            a0z -= g0.z;
            a0q = fmaf(xi.w, q0, a0q);
            a1x -= g1.x;
            a1y -= g1.y;
            a1z -= g1.z;
            a1q = fmaf(xi.w, q1, a1q);
            add_par<PRIV>(p6, p12, u0, lane, in0, c60, c120);
            add_par<PRIV>(p6, p12, u1, lane, in1, c61, c121);
        }
        int one = lo ^ hi;
#pragma unroll 1
        while (one) {
            const int k = __ffs(one) - 1;
            one &= one - 1;
            const bool upper = (hi >> k) & 1;  // warp-uniform
            const bool b = (mw >> (2 * k + (upper ? 1 : 0))) & 1u;
            const float4 xj = upper ? xj1 : xj0, gj = upper ? gj1 : gj0;
            const int tb = upper ? tb1 : tb0;
            const float4 xi = s_xi[k * NB_CL + ti];
            const float4 gi = s_gi[k * NB_CL + ti];
            const int ta = s_ti[k * NB_CL + ti];
            float3 g;
            float q, c6, c12;
            int u;
            const bool in = vjp_pair<COUL>(v, lje, make_float3(xi.x - xj.x, xi.y - xj.y, xi.z - xj.z),
                                           make_float3(gi.x - gj.x, gi.y - gj.y, gi.z - gj.z), xi.w, xj.w, ta * T + tb,
                                           b, gE, g, q, c6, c12, u);
            float *ga = s_ga + k * 128 + lane;
            ga[0] += g.x;
            ga[32] += g.y;
            ga[64] += g.z;
            ga[96] += xj.w * q;
            if (upper) {
                a1x -= g.x;
                a1y -= g.y;
                a1z -= g.z;
                a1q = fmaf(xi.w, q, a1q);
            } else {
                a0x -= g.x;
                a0y -= g.y;
                a0z -= g.z;
                a0q = fmaf(xi.w, q, a0q);
            }
            add_par<PRIV>(p6, p12, u, lane, in, c6, c12);
        }
        // j-gradients over the 8 i-lanes, transposed as in the force kernel
        const bool up = ti & 4;
        float kx = up ? a1x : a0x, ky = up ? a1y : a0y, kz = up ? a1z : a0z, kq = up ? a1q : a0q;
        kx += __shfl_xor_sync(full, up ? a0x : a1x, 4);
        ky += __shfl_xor_sync(full, up ? a0y : a1y, 4);
        kz += __shfl_xor_sync(full, up ? a0z : a1z, 4);
        kq += __shfl_xor_sync(full, up ? a0q : a1q, 4);
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
            kx += __shfl_xor_sync(full, kx, o);
            ky += __shfl_xor_sync(full, ky, o);
            kz += __shfl_xor_sync(full, kz, o);
            kq += __shfl_xor_sync(full, kq, o);
        }
        if ((ti & 3) == 0) {
            const int sj = cj * NB_CL + tj + (up ? 4 : 0);
            atomicAdd(&v.gx[sj], make_float4(kx, ky, kz, 0.f));
            atomicAdd(&v.gq[sj], kq);
        }
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < NB_SCL; k++) {
        float gx = s_ga[k * 128 + lane], gy = s_ga[k * 128 + 32 + lane], gz = s_ga[k * 128 + 64 + lane];
        float gq = s_ga[k * 128 + 96 + lane];
        for (int o = 8; o < 32; o <<= 1) {
            gx += __shfl_xor_sync(full, gx, o);
            gy += __shfl_xor_sync(full, gy, o);
            gz += __shfl_xor_sync(full, gz, o);
            gq += __shfl_xor_sync(full, gq, o);
        }
        if (tj == 0) {
            atomicAdd(&v.gx[si * NB_SCA + k * NB_CL + ti], make_float4(gx, gy, gz, 0.f));
            atomicAdd(&v.gq[si * NB_SCA + k * NB_CL + ti], gq);
        }
    }
}

// Persistent: each warp takes its first item by index and later ones from the
// context's counter (zeroed by the gather); parameter accumulators are folded
// into the FP64 table after each item.
template <int COUL, bool PRIV>
__global__ void __launch_bounds__(kVW * 32) k_vjp(VjpView v, int *queue) {
    __shared__ float4 s_xi[kVW][NB_SCA];
    __shared__ float4 s_gi[kVW][NB_SCA];
    __shared__ int s_ti[kVW][NB_SCA];
    __shared__ float s_ga[kVW][4 * NB_SCL * 32];
    __shared__ float4 s_lje[kVjpMaxT * kVjpMaxT];
    __shared__ int s_ord[kVjpMaxT * (kVjpMaxT + 1) / 2];
    // parameter accumulators per unordered type pair {a, b} (a <= b), index
    // u = a T - a (a - 1) / 2 + b - a; PRIV: [kVW][2][TS][33]; else [kVW][2][TS]
    extern __shared__ float s_par[];
    const SysView &sv = v.s;
    const int T = sv.T, TT = T * T, TS = T * (T + 1) / 2;
    for (int t = threadIdx.x; t < TT; t += blockDim.x) {
        const int a = min(t / T, t % T), b = max(t / T, t % T);
        const int u = a * T - a * (a - 1) / 2 + b - a;
        float4 le = sv.lje[t];
        le.w = __int_as_float(u);  // the pair's accumulator, read with its parameters
        s_lje[t] = le;
        if (a == t / T) s_ord[u] = t;  // a <= b: the slot gpar[a T + b] receives the pair's total
    }
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned full = 0xffffffffu;
    float *const p6 = s_par + (size_t)wib * 2 * TS * (PRIV ? kColStride : 1);
    float *const p12 = p6 + TS * (PRIV ? kColStride : 1);
    if (PRIV) {
        for (int t = 0; t < TS; t++) {
            p6[t * kColStride + lane] = 0.f;
            p12[t * kColStride + lane] = 0.f;
        }
    } else {
        for (int t = lane; t < TS; t += 32) {
            p6[t] = 0.f;
            p12[t] = 0.f;
        }
    }
    __syncthreads();
    const int n_warps = gridDim.x * kVW;
    const float gE = v.gE_dev ? (float)*v.gE_dev : v.gE;
    int w = blockIdx.x * kVW + wib;
    while (w < sv.n_items) {
        const int nj = sv.inner_len[w];
        if (nj > 0) {
            vjp_item<COUL, PRIV>(v, w, nj, s_xi[wib], s_gi[wib], s_ti[wib], s_ga[wib], s_lje, p6, p12, T, gE);
            __syncwarp();
            for (int t = lane; t < TS; t += 32) {
                float a = 0.f, b = 0.f;
                if (PRIV) {  // lane t folds row t over the 32 lane columns (banks (t + l) mod 32), then clears it
                    for (int l = 0; l < 32; l++) {
                        a += p6[t * kColStride + l];
                        b += p12[t * kColStride + l];
                        p6[t * kColStride + l] = 0.f;
                        p12[t * kColStride + l] = 0.f;
                    }
                } else {
                    a = p6[t];
                    b = p12[t];
                    p6[t] = 0.f;
                    p12[t] = 0.f;
                }
                // the total of the unordered pair into one ordered slot; the finish kernel
                // symmetrises (gpar[a T + b] + gpar[b T + a]) / 2
                if (a != 0.f) atomicAdd(&v.gpar[s_ord[t]], (double)a);
                if (b != 0.f) atomicAdd(&v.gpar[TT + s_ord[t]], (double)b);
            }
        }
        __syncwarp();  // the staging arrays and accumulators are reused by the next item
        int claim = 0;
        if (lane == 0) claim = atomicAdd(queue, 1);
        w = n_warps + __shfl_sync(full, claim, 0);
    }
}

__global__ void k_vjp_gather(int nslots, const int *__restrict__ perm, const float *__restrict__ x,
                             const int *__restrict__ img, const float *__restrict__ q_s,
                             const float *__restrict__ gF, double Lx, double Ly, double Lz, float4 *__restrict__ xq,
                             float4 *__restrict__ gf, float4 *__restrict__ gx, float *__restrict__ gq, double *gpar,
                             int n_par, int *err, int *queue) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0) *queue = 0;
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
void launch_vjp(const VjpView &v, int nb, size_t smem, int n_sm, int *queue, cudaStream_t st) {
    // the default limit of 48 KB covers static and dynamic shared memory together
    if (smem > 16 * 1024) cudaFuncSetAttribute(k_vjp<COUL, PRIV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_vjp<COUL, PRIV>, kVW * 32, smem) != cudaSuccess || occ < 1)
        occ = 1;
    k_vjp<COUL, PRIV><<<std::min(nb, std::max(n_sm, 1) * occ), kVW * 32, smem, st>>>(v, queue);
}

}  // namespace

nb_status nb_launch_vjp(nb_ctx *c, const float *x, const float *gF, double gE, const double *gE_dev, float *gx,
                        float *gq, double *gc6, double *gc12, cudaStream_t st) {
    if (c->T > kVjpMaxT) return NB_ERR_INVALID_ARG;
    const int ns = c->S_host * NB_SCA;
    const int npar = 2 * c->T * c->T;
    const int nthr = ns > npar ? ns : npar;
    c->xq_cur = nullptr;  // the adjoint gathers its positions into the context's own array
    k_vjp_gather<<<(nthr + 255) / 256, 256, 0, st>>>(ns, c->perm, x, c->img, c->q_s, gF, c->box[0], c->box[1],
                                                      c->box[2], c->xq, c->gfs, c->gxs, c->gqs, c->gpar, npar,
                                                      c->err, c->queue);
    VjpView v;
    v.s = nb_make_view(c, c->fs, nullptr, nullptr);
    v.gf = c->gfs;
    v.gx = c->gxs;
    v.gq = c->gqs;
    v.gpar = c->gpar;
    v.gE = (float)gE;
    v.gE_dev = gE_dev;
    v.two_beta_sqrtpi = (float)(2.0 * c->beta / sqrt(M_PI));
    c->n_launches += 2;
    if (v.s.n_items > 0) {
        NbTraceScope tr(c, NB_TRACE_VJP, st);
        c->n_launches++;
        const int nb = (v.s.n_items + kVW - 1) / kVW;
        const int TS = c->T * (c->T + 1) / 2;
        if (c->T <= kVjpPrivMaxT) {
            const size_t smem = sizeof(float) * kVW * 2 * TS * kColStride;
            if (c->coulomb == NB_COULOMB_RF)
                launch_vjp<NB_COULOMB_RF, true>(v, nb, smem, c->n_sm, c->queue, st);
            else if (c->coulomb == NB_COULOMB_EWALD)
                launch_vjp<NB_COULOMB_EWALD, true>(v, nb, smem, c->n_sm, c->queue, st);
            else
                launch_vjp<NB_COULOMB_NONE, true>(v, nb, smem, c->n_sm, c->queue, st);
        } else {
            const size_t smem = sizeof(float) * kVW * 2 * TS;
            if (c->coulomb == NB_COULOMB_RF)
                launch_vjp<NB_COULOMB_RF, false>(v, nb, smem, c->n_sm, c->queue, st);
            else if (c->coulomb == NB_COULOMB_EWALD)
                launch_vjp<NB_COULOMB_EWALD, false>(v, nb, smem, c->n_sm, c->queue, st);
            else
                launch_vjp<NB_COULOMB_NONE, false>(v, nb, smem, c->n_sm, c->queue, st);
        }
    }
    const int nf = c->N > c->T * c->T ? c->N : c->T * c->T;
    k_vjp_finish<<<(nf + 255) / 256, 256, 0, st>>>(c->N, c->inv, c->gxs, c->gqs, gx, gq, c->T, c->gpar, gc6, gc12);
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}
