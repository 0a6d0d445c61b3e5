// Reciprocal-space Ewald by smooth PME, and the exclusion and self terms that
// complete the Ewald sum together with the short-range kernel.
//
// The paper runs PME as its own GPU task on a separate stream, dominated by two
// 3-D FFTs on small grids (Sec. IV), and computes the real-space part in the
// non-bonded kernel (Sec. V.A).  The method is smooth PME (cardinal B-spline
// charge assignment, FFT, influence function, FFT back, B-spline gradient
// gather).  Layout: one FP32 charge grid K1 x K2 x K3 (K3 fastest), its R2C
// transform K1 x K2 x (K3/2+1); cuFFT does the two transforms.  Fractional
// coordinates are formed in FP64 (a 25 nm box on a 200-point grid would lose
// five bits of the B-spline argument in FP32); weights, grid and gather are FP32,
// the energy and virial sums FP64, and the Coulomb constant is applied once in
// FP64 to the energies.
#include <cufft.h>
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "nb_pair.cuh"

using namespace nbk;

struct nb_pme {
    int n = 0, order = 0;
    int K[3] = {0, 0, 0};
    double beta = 0, eps_r = 1;
    float *grid = nullptr;       // [K1*K2*K3] real grid (charges, then the convolution)
    cufftComplex *cgrid = nullptr;  // [K1*K2*(K3/2+1)]
    float *bsp = nullptr;        // [K1+K2+K3] B-spline moduli |b(m)|^2 per axis
    double *acc = nullptr;       // [7] energy and virial sums of the solve (without f)
    cufftHandle fwd = 0, bwd = 0;
    bool have_fwd = false, have_bwd = false;
};

namespace {

constexpr int kPmeMaxOrder = 8;

// M_n(w + j), j = 0..n-1 (cardinal B-spline of order n at the n grid offsets of
// an atom with fractional part w), and d/dw of the same.  Built from the order-2
// spline by the recursion M_k(u) = (u M_{k-1}(u) + (k - u) M_{k-1}(u - 1)) / (k - 1),
// in place from the highest offset down.
template <int N>
__device__ __forceinline__ void bspline_weights(float w, float (&th)[N], float (&dth)[N]) {
#pragma unroll
    for (int j = 0; j < N; j++) th[j] = 0.f;
    th[0] = w;
    th[1] = 1.f - w;
#pragma unroll
    for (int k = 3; k <= N; k++) {
        if (k == N) {
            // derivative of M_N at w + j: M_{N-1}(w + j) - M_{N-1}(w + j - 1)
            dth[0] = th[0];
#pragma unroll
            for (int j = 1; j < N; j++) dth[j] = th[j] - th[j - 1];
        }
        const float inv = 1.f / (float)(k - 1);
#pragma unroll
        for (int j = k - 1; j >= 1; j--) th[j] = ((w + j) * th[j] + ((float)k - w - j) * th[j - 1]) * inv;
        th[0] = w * th[0] * inv;
    }
}

struct PmeGeom {
    int K[3];
    double kl[3];  // K_a / L_a
};

// Base grid index in [0, K) and fractional part of coordinate x on one axis
// (FP64).  False for a non-finite coordinate (the atom is then skipped).
__device__ __forceinline__ bool frac_coord(float x, int K, double kl, int &fl, float &w) {
    if (!isfinite(x)) return false;
    double u = (double)x * kl;
    u -= (double)K * floor(u / (double)K);  // [0, K] up to rounding, which may leave -ulp or K
    int f = (int)floor(u);
    const double fr = u - (double)f;
    if (f < 0) f += K;
    if (f >= K) f -= K;
    fl = min(max(f, 0), K - 1);
    w = (float)fr;
    return true;
}

// Charge spreading: ORDER threads per atom, thread j0 adds the ORDER x ORDER
// weights of its x-plane; consecutive z offsets are neighbouring addresses.
template <int ORDER>
__global__ void k_pme_spread(int n, const float *__restrict__ x, const float *__restrict__ q, PmeGeom g,
                             float *__restrict__ grid) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(t / ORDER), j0 = (int)(t % ORDER);
    if (i >= n) return;
    const float qi = q[i];
    if (qi == 0.f) return;
    float th[3][ORDER], dth[ORDER];
    int fl[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float w = 0.f;
        ok &= frac_coord(x[3 * i + a], g.K[a], g.kl[a], fl[a], w);
        bspline_weights<ORDER>(w, th[a], dth);
    }
    if (!ok) return;
    int i0 = fl[0] - j0;
    if (i0 < 0) i0 += g.K[0];
    float t0 = 0.f;  // this thread's x-plane weight, selected without a dynamic index
#pragma unroll
    for (int j = 0; j < ORDER; j++) t0 = (j == j0) ? th[0][j] : t0;
    t0 *= qi;
#pragma unroll
    for (int j1 = 0; j1 < ORDER; j1++) {
        int i1 = fl[1] - j1;
        if (i1 < 0) i1 += g.K[1];
        const float t01 = t0 * th[1][j1];
        float *row = grid + ((size_t)i0 * g.K[1] + i1) * g.K[2];
#pragma unroll
        for (int j2 = 0; j2 < ORDER; j2++) {
            int i2 = fl[2] - j2;
            if (i2 < 0) i2 += g.K[2];
            atomicAdd(row + i2, t01 * th[2][j2]);
        }
    }
}

// Influence function on the half spectrum: multiply each coefficient by
// B(m) C(m) and sum the energy and virial terms (FP64; the Coulomb constant is
// applied later).  Coefficients with 0 < m3 < K3/2 stand for two (m, -m).
__global__ void k_pme_solve(cufftComplex *__restrict__ cg, int K1, int K2, int K3, float L0, float L1, float L2,
                            float beta, const float *__restrict__ bsp, double *__restrict__ acc) {
    const int K3h = K3 / 2 + 1;
    const long long total = (long long)K1 * K2 * K3h;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0, w[6] = {0, 0, 0, 0, 0, 0};
    if (idx < total) {
        const int i2 = (int)(idx % K3h);
        const int i1 = (int)((idx / K3h) % K2);
        const int i0 = (int)(idx / ((long long)K3h * K2));
        const float mx = (float)(i0 <= K1 / 2 ? i0 : i0 - K1) / L0;
        const float my = (float)(i1 <= K2 / 2 ? i1 : i1 - K2) / L1;
        const float mz = (float)i2 / L2;
        const float m2 = mx * mx + my * my + mz * mz;
        float eterm = 0.f;
        if (idx != 0) {
            const float pi = 3.14159265358979f;
            const float V = L0 * L1 * L2;
            eterm = expf(-pi * pi * m2 / (beta * beta)) / (pi * V * m2) * bsp[i0] * bsp[K1 + i1] * bsp[K1 + K2 + i2];
            const cufftComplex d = cg[idx];
            const float s2 = d.x * d.x + d.y * d.y;
            const float wgt = (i2 == 0 || (K3 % 2 == 0 && i2 == K3 / 2)) ? 1.f : 2.f;
            const double ek = 0.5 * (double)wgt * (double)eterm * (double)s2;
            e = ek;
            const double g2 = 2.0 * (1.0 + (double)(pi * pi * m2 / (beta * beta))) / (double)m2;
            const double m[3] = {mx, my, mz};
            // xx, yy, zz, xy, xz, yz of -1/2 e (delta - g2 m m)
            w[0] = -0.5 * ek * (1.0 - g2 * m[0] * m[0]);
            w[1] = -0.5 * ek * (1.0 - g2 * m[1] * m[1]);
            w[2] = -0.5 * ek * (1.0 - g2 * m[2] * m[2]);
            w[3] = 0.5 * ek * g2 * m[0] * m[1];
            w[4] = 0.5 * ek * g2 * m[0] * m[2];
            w[5] = 0.5 * ek * g2 * m[1] * m[2];
        }
        cufftComplex d = cg[idx];
        d.x *= eterm;
        d.y *= eterm;
        cg[idx] = d;
    }
    // block reduction of the 7 sums, then one atomic per sum per block
    __shared__ double s_red[7][32];
    const unsigned full = 0xffffffffu;
    double v[7] = {e, w[0], w[1], w[2], w[3], w[4], w[5]};
#pragma unroll
    for (int k = 0; k < 7; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(full, v[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 7; k++) s_red[k][wid] = v[k];
    __syncthreads();
    if (threadIdx.x < 7) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) s += s_red[threadIdx.x][k];
        atomicAdd(&acc[threadIdx.x], s);
    }
}

// Energy and virial out (times the Coulomb constant), accumulators zeroed.
__global__ void k_pme_finish(double *acc, double fc, double *e, double *vir) {
    if (threadIdx.x != 0) return;
    if (e) e[0] = fc * acc[0];
    if (vir) {
        const double xx = acc[1], yy = acc[2], zz = acc[3], xy = acc[4], xz = acc[5], yz = acc[6];
        const double W[9] = {xx, xy, xz, xy, yy, yz, xz, yz, zz};
        for (int k = 0; k < 9; k++) vir[k] = fc * W[k];
    }
    for (int k = 0; k < 7; k++) acc[k] = 0.0;
}

// Force gather: one thread per atom, F_i = -f q_i sum_k grad(weights) conv(k).
template <int ORDER>
__global__ void k_pme_gather(int n, const float *__restrict__ x, const float *__restrict__ q, PmeGeom g,
                             const float *__restrict__ conv, float fcoul, float *__restrict__ f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float qi = q[i];
    if (qi == 0.f) return;
    float th[3][ORDER], dth[3][ORDER];
    int fl[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float w = 0.f;
        ok &= frac_coord(x[3 * i + a], g.K[a], g.kl[a], fl[a], w);
        bspline_weights<ORDER>(w, th[a], dth[a]);
    }
    if (!ok) return;
    float fx = 0.f, fy = 0.f, fz = 0.f;
#pragma unroll
    for (int j0 = 0; j0 < ORDER; j0++) {
        int i0 = fl[0] - j0;
        if (i0 < 0) i0 += g.K[0];
#pragma unroll
        for (int j1 = 0; j1 < ORDER; j1++) {
            int i1 = fl[1] - j1;
            if (i1 < 0) i1 += g.K[1];
            const float *row = conv + ((size_t)i0 * g.K[1] + i1) * g.K[2];
            float s = 0.f, sd = 0.f;
#pragma unroll
            for (int j2 = 0; j2 < ORDER; j2++) {
                int i2 = fl[2] - j2;
                if (i2 < 0) i2 += g.K[2];
                const float v = row[i2];
                s = fmaf(th[2][j2], v, s);
                sd = fmaf(dth[2][j2], v, sd);
            }
            fx = fmaf(dth[0][j0] * th[1][j1], s, fx);
            fy = fmaf(th[0][j0] * dth[1][j1], s, fy);
            fz = fmaf(th[0][j0] * th[1][j1], sd, fz);
        }
    }
    const float c = -fcoul * qi;
    f[3 * i] += c * fx * (float)g.kl[0];
    f[3 * i + 1] += c * fy * (float)g.kl[1];
    f[3 * i + 2] += c * fz * (float)g.kl[2];
}

template <int ORDER>
void launch_spread_gather(nb_pme *p, bool gather, const float *x, const float *q, const PmeGeom &g, float fcoul,
                          float *f, cudaStream_t st) {
    if (!gather) {
        const long long threads = (long long)p->n * ORDER;
        k_pme_spread<ORDER><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(p->n, x, q, g, p->grid);
    } else {
        k_pme_gather<ORDER><<<(p->n + 127) / 128, 128, 0, st>>>(p->n, x, q, g, p->grid, fcoul, f);
    }
}

void dispatch_spread_gather(nb_pme *p, bool gather, const float *x, const float *q, const PmeGeom &g, float fcoul,
                            float *f, cudaStream_t st) {
    switch (p->order) {
        case 3: launch_spread_gather<3>(p, gather, x, q, g, fcoul, f, st); break;
        case 4: launch_spread_gather<4>(p, gather, x, q, g, fcoul, f, st); break;
        case 5: launch_spread_gather<5>(p, gather, x, q, g, fcoul, f, st); break;
        case 6: launch_spread_gather<6>(p, gather, x, q, g, fcoul, f, st); break;
        case 7: launch_spread_gather<7>(p, gather, x, q, g, fcoul, f, st); break;
        default: launch_spread_gather<8>(p, gather, x, q, g, fcoul, f, st); break;
    }
}

// |b(m)|^2 = 1 / |sum_{k=0}^{n-2} M_n(k+1) exp(2 pi i m k / K)|^2 (host, FP64); where an
// odd order makes the sum vanish (m = K/2) the mean of the neighbours is used.
std::vector<double> bspline_moduli(int K, int order) {
    // M_n at the integers 1..n-1 by the same recursion, in FP64
    std::vector<double> m(order + 1, 0.0), t(order + 1, 0.0);
    m[1] = 1.0;  // M_2(1) = 1 (M_2 at integers: 0, 1, 0)
    for (int k = 3; k <= order; k++) {
        for (int u = 0; u <= k; u++) {
            const double a = (u >= 0 && u <= k - 1) ? m[u] : 0.0;
            const double b = (u - 1 >= 0 && u - 1 <= k - 1) ? m[u - 1] : 0.0;
            t[u] = (u * a + (k - u) * b) / (k - 1);
        }
        m = t;
    }
    std::vector<double> out(K), den(K);
    for (int mm = 0; mm < K; mm++) {
        double re = 0.0, im = 0.0;
        for (int k = 0; k <= order - 2; k++) {
            const double ph = 2.0 * M_PI * mm * k / K;
            re += m[k + 1] * cos(ph);
            im += m[k + 1] * sin(ph);
        }
        den[mm] = re * re + im * im;
    }
    for (int mm = 0; mm < K; mm++) out[mm] = den[mm] > 1e-7 ? 1.0 / den[mm] : -1.0;
    for (int mm = 0; mm < K; mm++)
        if (out[mm] < 0) out[mm] = 0.5 * (1.0 / std::max(den[(mm + K - 1) % K], 1e-7) + 1.0 / std::max(den[(mm + 1) % K], 1e-7));
    return out;
}

// Exclusion and self terms (one thread per atom, all partners in the symmetric
// CSR): V = -f qi qj erf(beta r)/r per excluded pair, whose force is
// -f qi qj beta^3 H(beta r) r_vec with the same H as the force kernel (no
// cancellation at small r); energies and virial of each pair are taken by the
// lower index, forces by both atoms (no atomics).  Self: -f beta/sqrt(pi) q^2.
__global__ void k_ewald_corr(int n, const float *__restrict__ x, const float *__restrict__ q,
                             const int *__restrict__ off, const int *__restrict__ idx, float Lx, float Ly, float Lz,
                             float beta, double beta_d, float ew_s, float fcoul, float *__restrict__ f,
                             double *__restrict__ acc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // E_excl, E_self, xx, yy, zz, xy, xz, yz (without f)
    if (i < n) {
        const float qi = q[i];
        const float xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
        const float b3 = beta * beta * beta;
        float fx = 0.f, fy = 0.f, fz = 0.f;
        for (int p = off[i]; p < off[i + 1]; p++) {
            const int j = idx[p];
            const float qq = qi * q[j];
            float dx = xi - x[3 * j], dy = yi - x[3 * j + 1], dz = zi - x[3 * j + 2];
            dx -= Lx * rintf(dx / Lx);
            dy -= Ly * rintf(dy / Ly);
            dz -= Lz * rintf(dz / Lz);
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float r = sqrtf(r2);
            const float z = beta * r;
            float h;
            if (z < (float)NB_EW_ZMAX_D) {
                h = ew_h(r2 * ew_s);
            } else {
                h = (erff(z) / z - 1.1283791670955126f * expf(-z * z)) / (z * z);
            }
            const float phi = -qq * b3 * h;  // force on i = f phi r_vec
            fx = fmaf(phi, dx, fx);
            fy = fmaf(phi, dy, fy);
            fz = fmaf(phi, dz, fz);
            if (j > i) {
                const double vij = r2 > 0.f ? -(double)qq * (double)erff(z) / (double)r
                                            : -(double)qq * 1.1283791670955126 * (double)beta;
                v[0] += vij;
                const double pd = (double)phi;
                v[2] += -0.5 * pd * dx * dx;
                v[3] += -0.5 * pd * dy * dy;
                v[4] += -0.5 * pd * dz * dz;
                v[5] += -0.5 * pd * dx * dy;
                v[6] += -0.5 * pd * dx * dz;
                v[7] += -0.5 * pd * dy * dz;
            }
        }
        v[1] = -beta_d * 0.5641895835477563 * (double)qi * (double)qi;
        f[3 * i] += fcoul * fx;
        f[3 * i + 1] += fcoul * fy;
        f[3 * i + 2] += fcoul * fz;
    }
    __shared__ double s_red[8][32];
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int k = 0; k < 8; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(full, v[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 8; k++) s_red[k][wid] = v[k];
    __syncthreads();
    if (threadIdx.x < 8) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) s += s_red[threadIdx.x][k];
        atomicAdd(&acc[threadIdx.x], s);
    }
}

__global__ void k_ewald_corr_finish(double *acc, double fc, double *e, double *vir) {
    if (threadIdx.x != 0) return;
    if (e) {
        e[0] = fc * acc[0];
        e[1] = fc * acc[1];
    }
    if (vir) {
        const double xx = acc[2], yy = acc[3], zz = acc[4], xy = acc[5], xz = acc[6], yz = acc[7];
        const double W[9] = {xx, xy, xz, xy, yy, yz, xz, yz, zz};
        for (int k = 0; k < 9; k++) vir[k] = fc * W[k];
    }
    for (int k = 0; k < 8; k++) acc[k] = 0.0;
}

bool box_ok(const double *box) {
    if (!box) return false;
    for (int a = 0; a < 3; a++)
        if (!(box[a] > 0.0) || !isfinite(box[a])) return false;
    return true;
}

}  // namespace

extern "C" {

nb_status nb_pme_create(const nb_pme_params *pp, nb_pme **out) {
    if (!pp || !out) return NB_ERR_INVALID_ARG;
    *out = nullptr;
    if (pp->n_atoms < 1 || pp->order < 3 || pp->order > kPmeMaxOrder || pp->reserved != 0) return NB_ERR_INVALID_ARG;
    for (int a = 0; a < 3; a++)
        if (pp->grid[a] < 2 * pp->order || pp->grid[a] > 4096) return NB_ERR_INVALID_ARG;
    if (!(pp->beta > 0.0) || !isfinite(pp->beta) || !(pp->eps_r > 0.0) || !isfinite(pp->eps_r))
        return NB_ERR_INVALID_ARG;
    nb_pme *p = new (std::nothrow) nb_pme;
    if (!p) return NB_ERR_CAPACITY;
    p->n = pp->n_atoms;
    p->order = pp->order;
    for (int a = 0; a < 3; a++) p->K[a] = pp->grid[a];
    p->beta = pp->beta;
    p->eps_r = pp->eps_r;
    const size_t nr = (size_t)p->K[0] * p->K[1] * p->K[2];
    const size_t nc = (size_t)p->K[0] * p->K[1] * (p->K[2] / 2 + 1);
    cudaError_t e = cudaMalloc((void **)&p->grid, sizeof(float) * nr);
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->cgrid, sizeof(cufftComplex) * nc);
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->bsp, sizeof(float) * (p->K[0] + p->K[1] + p->K[2]));
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->acc, sizeof(double) * 8);
    if (e == cudaSuccess) e = cudaMemset(p->acc, 0, sizeof(double) * 8);
    if (e == cudaSuccess) {
        std::vector<float> b;
        for (int a = 0; a < 3; a++) {
            const std::vector<double> m = bspline_moduli(p->K[a], p->order);
            for (double v : m) b.push_back((float)v);
        }
        e = cudaMemcpy(p->bsp, b.data(), sizeof(float) * b.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        nb_pme_destroy(p);
        return nb_cuda_status(e);
    }
    if (cufftPlan3d(&p->fwd, p->K[0], p->K[1], p->K[2], CUFFT_R2C) != CUFFT_SUCCESS) {
        nb_pme_destroy(p);
        return NB_ERR_CUDA;
    }
    p->have_fwd = true;
    if (cufftPlan3d(&p->bwd, p->K[0], p->K[1], p->K[2], CUFFT_C2R) != CUFFT_SUCCESS) {
        nb_pme_destroy(p);
        return NB_ERR_CUDA;
    }
    p->have_bwd = true;
    *out = p;
    return NB_OK;
}

void nb_pme_destroy(nb_pme *p) {
    if (!p) return;
    if (p->have_fwd) cufftDestroy(p->fwd);
    if (p->have_bwd) cufftDestroy(p->bwd);
    cudaFree(p->grid);
    cudaFree(p->cgrid);
    cudaFree(p->bsp);
    cudaFree(p->acc);
    delete p;
}

nb_status nb_pme_forces(nb_pme *p, unsigned flags, const float *x_dev, const float *q_dev, const double *box_host,
                        float *f_dev, double *e_dev, double *vir_dev, void *stream) {
    if (!p || !x_dev || !q_dev || !f_dev || !box_ok(box_host)) return NB_ERR_INVALID_ARG;
    if ((flags & ~(unsigned)(NB_ENERGY | NB_VIRIAL)) != 0) return NB_ERR_INVALID_ARG;
    if ((flags & NB_ENERGY) && !e_dev) return NB_ERR_INVALID_ARG;
    if ((flags & NB_VIRIAL) && !vir_dev) return NB_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    PmeGeom g;
    for (int a = 0; a < 3; a++) {
        g.K[a] = p->K[a];
        g.kl[a] = (double)p->K[a] / box_host[a];
    }
    const size_t nr = (size_t)p->K[0] * p->K[1] * p->K[2];
    const size_t nc = (size_t)p->K[0] * p->K[1] * (p->K[2] / 2 + 1);
    const float fcoul = (float)(138.935458 / p->eps_r);
    NB_CUDA_TRY(cudaMemsetAsync(p->grid, 0, sizeof(float) * nr, st));
    dispatch_spread_gather(p, false, x_dev, q_dev, g, fcoul, f_dev, st);
    NB_CUDA_TRY(cudaGetLastError());
    if (cufftSetStream(p->fwd, st) != CUFFT_SUCCESS || cufftExecR2C(p->fwd, p->grid, p->cgrid) != CUFFT_SUCCESS)
        return NB_ERR_CUDA;
    k_pme_solve<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(p->cgrid, p->K[0], p->K[1], p->K[2], (float)box_host[0],
                                                            (float)box_host[1], (float)box_host[2], (float)p->beta,
                                                            p->bsp, p->acc);
    NB_CUDA_TRY(cudaGetLastError());
    k_pme_finish<<<1, 32, 0, st>>>(p->acc, 138.935458 / p->eps_r, (flags & NB_ENERGY) ? e_dev : nullptr,
                                   (flags & NB_VIRIAL) ? vir_dev : nullptr);
    NB_CUDA_TRY(cudaGetLastError());
    if (cufftSetStream(p->bwd, st) != CUFFT_SUCCESS || cufftExecC2R(p->bwd, p->cgrid, p->grid) != CUFFT_SUCCESS)
        return NB_ERR_CUDA;
    dispatch_spread_gather(p, true, x_dev, q_dev, g, fcoul, f_dev, st);
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}

nb_status nb_ewald_corrections(nb_ctx *c, unsigned flags, const float *x_dev, float *f_dev, double *e_dev,
                               double *vir_dev, void *stream) {
    if (!c || !x_dev || !f_dev) return NB_ERR_INVALID_ARG;
    if (c->coulomb != NB_COULOMB_EWALD) return NB_ERR_INVALID_ARG;
    if ((flags & ~(unsigned)(NB_ENERGY | NB_VIRIAL)) != 0) return NB_ERR_INVALID_ARG;
    if ((flags & NB_ENERGY) && !e_dev) return NB_ERR_INVALID_ARG;
    if ((flags & NB_VIRIAL) && !vir_dev) return NB_ERR_INVALID_ARG;
    if (!c->have_grid) return NB_ERR_NOT_READY;  // the box comes from the last grid sort
    cudaStream_t st = (cudaStream_t)stream;
    const float ew_s = (float)(c->beta * c->beta / (NB_EW_ZMAX_D * NB_EW_ZMAX_D));
    c->n_launches += 2;
    k_ewald_corr<<<(c->N + 127) / 128, 128, 0, st>>>(c->N, x_dev, c->q, c->excl_off, c->excl_idx, (float)c->box[0],
                                                     (float)c->box[1], (float)c->box[2], (float)c->beta, c->beta, ew_s,
                                                     (float)(138.935458 / c->eps_r), f_dev, c->ewald_acc);
    NB_CUDA_TRY(cudaGetLastError());
    k_ewald_corr_finish<<<1, 32, 0, st>>>(c->ewald_acc, 138.935458 / c->eps_r, (flags & NB_ENERGY) ? e_dev : nullptr,
                                          (flags & NB_VIRIAL) ? vir_dev : nullptr);
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}

}  // extern "C"
