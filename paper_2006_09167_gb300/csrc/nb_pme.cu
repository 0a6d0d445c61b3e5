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
    int n = 0, order = 0, n_sm = 1;
    int K[3] = {0, 0, 0};
    double beta = 0, eps_r = 1;
    float *grid = nullptr;       // [K1*K2*K3] real grid (charges, then the convolution)
    cufftComplex *cgrid = nullptr;  // [K1*K2*(K3/2+1)]
    float *bsp = nullptr;        // [K1+K2+K3] B-spline moduli |b(m)|^2 per axis
    double *part = nullptr;      // [kRows*8] per-block energy and virial rows of the solve (without f)
    unsigned *count = nullptr;   // finished-block counter of the solve (zero between calls)
    cufftHandle fwd = 0, bwd = 0;
    bool have_fwd = false, have_bwd = false;
};

namespace {

constexpr int kPmeMaxOrder = 8;
constexpr int kRows = 1024;  // grid cap of the reducing kernels (rows of partial sums)

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
    float kl_hi[3], kl_lo[3];  // K_a / L_a as a float pair
};

// Base grid index in [0, K) and fractional part of coordinate x on one axis.
// u = x K/L is formed as a float pair (the product split exactly by an FMA, K/L
// itself a float pair), so the fractional part keeps ~1e-7 absolute accuracy
// however large u is; the whole part is reduced modulo K in integers.  False
// for a non-finite coordinate (the atom is then skipped).
__device__ __forceinline__ bool frac_coord(float x, int K, float kl_hi, float kl_lo, int &fl, float &w) {
    if (!isfinite(x)) return false;
    const float u_hi = x * kl_hi;
    const float u_lo = fmaf(x, kl_hi, -u_hi) + x * kl_lo;
    float fh = floorf(u_hi);
    float fr = (u_hi - fh) + u_lo;  // u_hi - fh is exact (|u_hi| < 2^24 for any sane box)
    if (fr < 0.f) {
        fr += 1.f;
        fh -= 1.f;
    } else if (fr >= 1.f) {
        fr -= 1.f;
        fh += 1.f;
    }
    if (!(fabsf(fh) < 1.6e7f)) return false;  // beyond exact integer range: treat as invalid input
    int f = (int)fh % K;
    if (f < 0) f += K;
    fl = min(max(f, 0), K - 1);
    w = fminf(fmaxf(fr, 0.f), 1.f);
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
        ok &= frac_coord(x[3 * i + a], g.K[a], g.kl_hi[a], g.kl_lo[a], fl[a], w);
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

// Block sum of NV per-thread values: value k is taken from d[] and summed in FP64
// throughout if bit k of D64 is set, else from a[] and summed in FP32 within a
// warp and FP64 across warps.  The block totals land in s_tot[0..NV) (shared
// memory), valid after the call in every thread.
template <int NV, unsigned D64>
__device__ void block_sum(const float (&a)[NV], const double (&d)[NV], double *s_tot) {
    __shared__ double s_red[8][32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double v;
        if (!((D64 >> k) & 1u)) {
            float x = a[k];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(full, x, o);
            v = (double)x;
        } else {
            v = d[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(full, v, o);
        }
        if (lane == 0) s_red[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_red[threadIdx.x][w];
        s_tot[threadIdx.x] = t;
    }
    __syncthreads();
}

// End of a two-stage reduction without a second launch: every block writes its
// row of NV totals (FP64); the last block to finish (a device counter, which that
// block resets) folds all rows in a fixed order and writes the outputs times the
// Coulomb constant fc.  Row layout: NE energies, then xx, yy, zz, xy, xz, yz.
// No block waits for another.
template <int NE>
__device__ void rows_out(const double *s_tot, double *__restrict__ part, unsigned *__restrict__ count, double fc,
                         double *e, double *vir) {
    constexpr int NV = NE + 6;
    __shared__ bool s_last;
    if (threadIdx.x < NV) part[(size_t)blockIdx.x * 8 + threadIdx.x] = s_tot[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(count, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the whole block folds the rows: strided partial sums, then a block sum
    double t[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) t[k] = 0.0;
    for (unsigned r = threadIdx.x; r < gridDim.x; r += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; k++) t[k] += __ldcg(part + (size_t)r * 8 + k);
    __shared__ double s_fold[NV][32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_xor_sync(full, t[k], o);
        if (lane == 0) s_fold[k][wid] = t[k];
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += s_fold[threadIdx.x][w];
        const int k = threadIdx.x;
        if (k < NE) {
            if (e) e[k] = fc * tot;
        } else if (vir) {
            const int c = k - NE;  // xx, yy, zz, xy, xz, yz -> row-major 3x3 slots
            const int ia = c < 3 ? 4 * c : (c == 3 ? 1 : (c == 4 ? 2 : 5));
            const int ib = c < 3 ? 4 * c : (c == 3 ? 3 : (c == 4 ? 6 : 7));
            vir[ia] = fc * tot;
            vir[ib] = fc * tot;
        }
    }
    if (threadIdx.x == 0) *count = 0u;
}

// Influence function on the half spectrum: multiply each coefficient by
// B(m) C(m) and sum the energy and virial terms (the Coulomb constant is applied
// at the end).  Coefficients with 0 < m3 < K3/2 stand for two (m, -m).  Each warp
// walks whole rows (i0, i1) of the half spectrum, lanes along i3; a capped grid.
__global__ void k_pme_solve(cufftComplex *__restrict__ cg, int K1, int K2, int K3, float L0, float L1, float L2,
                            float beta, const float *__restrict__ bsp, double *__restrict__ part,
                            unsigned *__restrict__ count, double fc, double *e, double *vir) {
    const int K3h = K3 / 2 + 1;
    const float pi = 3.14159265358979f;
    const float V = L0 * L1 * L2;
    const float pb2 = pi * pi / (beta * beta);
    const int lane = threadIdx.x & 31;
    const int warps = (int)(gridDim.x * blockDim.x) >> 5;
    float a[7] = {0, 0, 0, 0, 0, 0, 0};  // E, xx, yy, zz, xy, xz, yz of -1/2 e (delta - g2 m m)
    for (int r = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); r < K1 * K2; r += warps) {
        const int i0 = r / K2, i1 = r - i0 * K2;
        const float mx = (float)(i0 <= K1 / 2 ? i0 : i0 - K1) / L0;
        const float my = (float)(i1 <= K2 / 2 ? i1 : i1 - K2) / L1;
        const float bxy = bsp[i0] * bsp[K1 + i1];
        cufftComplex *row = cg + (size_t)r * K3h;
        for (int i2 = lane; i2 < K3h; i2 += 32) {
            const float mz = (float)i2 / L2;
            const float m2 = mx * mx + my * my + mz * mz;
            cufftComplex d = row[i2];
            float eterm = 0.f;
            if (r != 0 || i2 != 0) {
                eterm = __expf(-pb2 * m2) / (pi * V * m2) * bxy * bsp[K1 + K2 + i2];
                const float s2 = d.x * d.x + d.y * d.y;
                const float wgt = (i2 == 0 || (K3 % 2 == 0 && i2 == K3 / 2)) ? 0.5f : 1.f;
                const float ek = wgt * eterm * s2;
                const float h = ek * (1.f + pb2 * m2) / m2;  // 1/2 ek g2
                a[0] += ek;
                a[1] += fmaf(h * mx, mx, -0.5f * ek);
                a[2] += fmaf(h * my, my, -0.5f * ek);
                a[3] += fmaf(h * mz, mz, -0.5f * ek);
                a[4] += h * mx * my;
                a[5] += h * mx * mz;
                a[6] += h * my * mz;
            }
            d.x *= eterm;
            d.y *= eterm;
            row[i2] = d;
        }
    }
    __shared__ double s_tot[8];
    const double dz[7] = {0, 0, 0, 0, 0, 0, 0};
    block_sum<7, 0u>(a, dz, s_tot);
    rows_out<1>(s_tot, part, count, fc, e, vir);
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
        ok &= frac_coord(x[3 * i + a], g.K[a], g.kl_hi[a], g.kl_lo[a], fl[a], w);
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
    f[3 * i] += c * fx * g.kl_hi[0];
    f[3 * i + 1] += c * fy * g.kl_hi[1];
    f[3 * i + 2] += c * fz * g.kl_hi[2];
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
// lower index, forces by both atoms (no atomics).  Self: -f beta/sqrt(pi) q^2
// (summed in FP64).  A capped grid walks the atoms; partial sums {E_excl, E_self,
// xx, yy, zz, xy, xz, yz} are folded by the last block.
__global__ void k_ewald_corr(int n, const float *__restrict__ x, const float *__restrict__ q,
                             const int *__restrict__ off, const int *__restrict__ idx, float Lx, float Ly, float Lz,
                             float beta, double beta_d, float ew_s, float fcoul, float *__restrict__ f,
                             double *__restrict__ part, unsigned *__restrict__ count, double fc, double *e,
                             double *vir) {
    float a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double d[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const float b3 = beta * beta * beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float qi = q[i];
        const float xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
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
                a[0] += r2 > 0.f ? -qq * (erff(z) / r) : -qq * 1.1283791670955126f * beta;
                const float hp = -0.5f * phi;
                a[2] += hp * dx * dx;
                a[3] += hp * dy * dy;
                a[4] += hp * dz * dz;
                a[5] += hp * dx * dy;
                a[6] += hp * dx * dz;
                a[7] += hp * dy * dz;
            }
        }
        d[1] += -beta_d * 0.5641895835477563 * (double)qi * (double)qi;
        f[3 * i] += fcoul * fx;
        f[3 * i + 1] += fcoul * fy;
        f[3 * i + 2] += fcoul * fz;
    }
    __shared__ double s_tot[8];
    block_sum<8, 2u>(a, d, s_tot);
    rows_out<2>(s_tot, part, count, fc, e, vir);
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
    if ((long long)pp->grid[0] * pp->grid[1] * (pp->grid[2] / 2 + 1) >= (1ll << 31)) return NB_ERR_INVALID_ARG;
    if (!(pp->beta > 0.0) || !isfinite(pp->beta) || !(pp->eps_r > 0.0) || !isfinite(pp->eps_r))
        return NB_ERR_INVALID_ARG;
    nb_pme *p = new (std::nothrow) nb_pme;
    if (!p) return NB_ERR_CAPACITY;
    p->n = pp->n_atoms;
    p->order = pp->order;
    for (int a = 0; a < 3; a++) p->K[a] = pp->grid[a];
    p->beta = pp->beta;
    p->eps_r = pp->eps_r;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || p->n_sm < 1)
        p->n_sm = 1;
    const size_t nr = (size_t)p->K[0] * p->K[1] * p->K[2];
    const size_t nc = (size_t)p->K[0] * p->K[1] * (p->K[2] / 2 + 1);
    cudaError_t e = cudaMalloc((void **)&p->grid, sizeof(float) * nr);
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->cgrid, sizeof(cufftComplex) * nc);
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->bsp, sizeof(float) * (p->K[0] + p->K[1] + p->K[2]));
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->part, sizeof(double) * 8 * kRows);
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->count, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(p->count, 0, sizeof(unsigned));
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
    cudaFree(p->part);
    cudaFree(p->count);
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
        const double kl = (double)p->K[a] / box_host[a];
        g.K[a] = p->K[a];
        g.kl_hi[a] = (float)kl;
        g.kl_lo[a] = (float)(kl - (double)g.kl_hi[a]);
    }
    const size_t nr = (size_t)p->K[0] * p->K[1] * p->K[2];
    const size_t nc = (size_t)p->K[0] * p->K[1] * (p->K[2] / 2 + 1);
    const float fcoul = (float)(138.935458 / p->eps_r);
    NB_CUDA_TRY(cudaMemsetAsync(p->grid, 0, sizeof(float) * nr, st));
    dispatch_spread_gather(p, false, x_dev, q_dev, g, fcoul, f_dev, st);
    NB_CUDA_TRY(cudaGetLastError());
    if (cufftSetStream(p->fwd, st) != CUFFT_SUCCESS || cufftExecR2C(p->fwd, p->grid, p->cgrid) != CUFFT_SUCCESS)
        return NB_ERR_CUDA;
    // one warp per spectrum row (K1*K2 rows), at most kRows blocks of 8 warps
    const int sblocks = std::min((p->K[0] * p->K[1] + 7) / 8, std::min(2 * p->n_sm, kRows));
    k_pme_solve<<<sblocks, 256, 0, st>>>(p->cgrid, p->K[0], p->K[1], p->K[2], (float)box_host[0], (float)box_host[1],
                                         (float)box_host[2], (float)p->beta, p->bsp, p->part, p->count,
                                         138.935458 / p->eps_r, (flags & NB_ENERGY) ? e_dev : nullptr,
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
    c->n_launches += 1;
    const int blocks = std::min((c->N + 255) / 256, std::min(2 * std::max(c->n_sm, 1), kRows));
    k_ewald_corr<<<blocks, 256, 0, st>>>(c->N, x_dev, c->q, c->excl_off, c->excl_idx, (float)c->box[0],
                                         (float)c->box[1], (float)c->box[2], (float)c->beta, c->beta, ew_s,
                                         (float)(138.935458 / c->eps_r), f_dev, c->ewald_part, c->ewald_count,
                                         138.935458 / c->eps_r, (flags & NB_ENERGY) ? e_dev : nullptr,
                                         (flags & NB_VIRIAL) ? vir_dev : nullptr);
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}

}  // extern "C"
