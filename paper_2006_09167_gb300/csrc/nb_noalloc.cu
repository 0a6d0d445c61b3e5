// Allocation-free evaluation of one small system (no context, no pair list).
//
// Every other entry point works on a context whose device buffers are
// allocated by nb_create / nb_grid_sort / nb_pairlist_build.  Some callers
// cannot call cudaMalloc at all: code inside a framework whose device memory is
// owned by another allocator (a caching allocator or a pool reserved up front),
// code that is not allowed to allocate after its start-up, or latency-critical
// code that cannot afford cudaMalloc/cudaFree, which may synchronise the
// device.  nb_forces_small_noalloc serves them: the caller passes only inputs
// and outputs, and the kernel's scratch (wrapped positions and types, a status
// word, and per-block partial sums of the energies and the virial) lives in a
// file-scope static device array, so the call allocates nothing.
//
// Inputs that only the device can check (atom types, exclusion row lengths) are
// validated by the first kernel; an invalid atom sets the status word, and then
// every output of the call is NaN (forces, energies, virial) instead of a
// silently wrong number.
//
// The kernel is a variant of the cluster pair force kernel for systems small
// enough to evaluate all pairs: each thread owns one i-atom and walks a chunk
// of j-atoms staged in shared memory, with the same pair interaction code
// (pair_phi) and the same exact periodic-shift handling; i-forces are added to
// the output with atomics (each unordered pair is computed from both sides,
// energies and the virial take half of each).
#include <math.h>
#include <string.h>

#include <mutex>

#include "nb_pair.cuh"

using namespace nbk;

namespace {

constexpr int kNaThreads = 128;   // i-atoms per block
constexpr int kNaJSplit = 8;      // j-chunks per i-block (grid.y)
constexpr int kNaMaxBlocks = (NB_NOALLOC_MAX_ATOMS + kNaThreads - 1) / kNaThreads * kNaJSplit;
constexpr int kNaRow = 11;        // E_LJ, E_C, 9 virial components

// The scratch: wrapped positions (x, y, z, q) and types of up to
// NB_NOALLOC_MAX_ATOMS atoms, the status word (non-zero: an atom failed the
// input checks; cleared by every call before its first kernel), then one row of
// partial sums per block.  Every call overwrites the other parts it reads.
struct NaScratch {
    float4 xq[NB_NOALLOC_MAX_ATOMS];
    int type[NB_NOALLOC_MAX_ATOMS];
    int bad;
    double rows[kNaMaxBlocks * kNaRow];
};
static __device__ __align__(256) NaScratch g_na_scratch;

struct NaArgs {
    SysView v;  // constants only (rc2, Coulomb and Ewald parameters)
    float2 lj[NB_NOALLOC_MAX_TYPES * NB_NOALLOC_MAX_TYPES];
    float4 lje[NB_NOALLOC_MAX_TYPES * NB_NOALLOC_MAX_TYPES];
    int n, T;
    double L[3];
    float Lhi[3], Llo[3], half[3];
    double coul_fd;  // 138.935458 / eps_r
    const float *x;
    const float *q;
    const int *type;
    const int *excl_off, *excl_idx;
    float *f;
    double *e, *vir;
    NaScratch *scr;  // device address of g_na_scratch
};

// Wrap the positions into the box, copy charges and types, zero the forces, and
// check what the host cannot: each type must lie in [0, T) and each exclusion
// row must have 0..NB_MAX_EXCL entries (an atom's own partners are kept in
// registers by the force kernel, so a longer row cannot be honoured).
__global__ void k_na_prep(const NaArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int t = a.type[i];
    bool ok = t >= 0 && t < a.T;
    if (a.excl_off) {
        const int lo = a.excl_off[i], hi = a.excl_off[i + 1];
        ok = ok && lo >= 0 && hi >= lo && hi - lo <= NB_MAX_EXCL;
    }
    if (!ok) atomicOr(&a.scr->bad, 1);
    float w[3];
    for (int k = 0; k < 3; k++) {
        const float xs = a.x[3 * i + k];
        const double nd = floor((double)xs / a.L[k]);
        float wf = nd == 0.0 ? xs : (float)((double)xs - nd * a.L[k]);
        if ((double)wf >= a.L[k]) wf = 0.f;
        w[k] = wf;
        a.f[3 * i + k] = 0.f;
    }
    a.scr->xq[i] = make_float4(w[0], w[1], w[2], a.q[i]);
    a.scr->type[i] = ok ? t : 0;
}

template <int COUL, bool EN>
__global__ void __launch_bounds__(kNaThreads) k_na_forces(const NaArgs a) {
    __shared__ float4 s_xj[kNaThreads];
    __shared__ int s_tj[kNaThreads];
    __shared__ float2 s_lj[NB_NOALLOC_MAX_TYPES * NB_NOALLOC_MAX_TYPES];
    __shared__ float4 s_lje[NB_NOALLOC_MAX_TYPES * NB_NOALLOC_MAX_TYPES];
    __shared__ double s_red[kNaThreads / 32][kNaRow];
    const int i = blockIdx.x * kNaThreads + threadIdx.x;
    if (a.scr->bad) {  // some atom failed the input checks: every force is NaN
        if (blockIdx.y == 0 && i < a.n) a.f[3 * i] = a.f[3 * i + 1] = a.f[3 * i + 2] = __int_as_float(0x7fffffff);
        return;  // (uniform over the grid: no block reaches the barriers below)
    }
    for (int t = threadIdx.x; t < a.T * a.T; t += blockDim.x) {
        s_lj[t] = a.lj[t];
        s_lje[t] = a.lje[t];
    }
    const bool active = i < a.n;
    float4 xi = active ? a.scr->xq[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int ti = active ? a.scr->type[i] * a.T : 0;
    int ex[NB_MAX_EXCL];
    int nex = 0;
    if (active && a.excl_off) {
        for (int e = a.excl_off[i]; e < a.excl_off[i + 1] && nex < NB_MAX_EXCL; e++) ex[nex++] = a.excl_idx[e];
    }
    const float qi = EN ? xi.w : xi.w * a.v.coul_f;
    const int chunk = (a.n + kNaJSplit - 1) / kNaJSplit;
    const int j_begin = blockIdx.y * chunk, j_end = min(a.n, j_begin + chunk);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    KSum elj, ec;
    float vr[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int j0 = j_begin; j0 < j_end; j0 += kNaThreads) {
        __syncthreads();
        const int jl = j0 + threadIdx.x;
        if (jl < j_end) {
            s_xj[threadIdx.x] = a.scr->xq[jl];
            s_tj[threadIdx.x] = a.scr->type[jl];
        }
        __syncthreads();
        const int m = min(kNaThreads, j_end - j0);
        for (int t = 0; t < m; t++) {
            const int j = j0 + t;
            const float4 xj = s_xj[t];
            bool bit = active && j != i;
            for (int e = 0; e < nex; e++) bit = bit && ex[e] != j;
            // minimum image with the side near the upper face shifted (exact)
            float d[3];
            const float pi[3] = {xi.x, xi.y, xi.z}, pj[3] = {xj.x, xj.y, xj.z};
            for (int k = 0; k < 3; k++) {
                float dk = pi[k] - pj[k];
                if (dk > a.half[k]) dk = ((pi[k] - a.Lhi[k]) - pj[k]) - a.Llo[k];
                else if (dk < -a.half[k]) dk = (pi[k] - (pj[k] - a.Lhi[k])) + a.Llo[k];
                d[k] = dk;
            }
            float pe_lj = 0.f, pe_c = 0.f;
            const float phi = pair_phi<COUL, EN>(a.v, s_lj, s_lje, make_float3(d[0], d[1], d[2]), qi, xj.w,
                                                 ti + s_tj[t], bit, pe_lj, pe_c);
            fx = fmaf(phi, d[0], fx);
            fy = fmaf(phi, d[1], fy);
            fz = fmaf(phi, d[2], fz);
            if (EN) {
                elj.add(0.5f * pe_lj);
                ec.add(0.5f * pe_c);
                for (int r = 0; r < 3; r++)
                    for (int c = 0; c < 3; c++) vr[3 * r + c] = fmaf(d[r] * phi, d[c], vr[3 * r + c]);
            }
        }
    }
    if (active) {
        atomicAdd(&a.f[3 * i], fx);
        atomicAdd(&a.f[3 * i + 1], fy);
        atomicAdd(&a.f[3 * i + 2], fz);
    }
    if (EN) {
        // block partial sums in FP64, one row per block
        double vals[kNaRow];
        vals[0] = (double)elj.s - (double)elj.c;
        vals[1] = (double)ec.s - (double)ec.c;
        for (int k = 0; k < 9; k++) vals[2 + k] = vr[k];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int k = 0; k < kNaRow; k++) {
            double s = vals[k];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) s_red[w][k] = s;
        }
        __syncthreads();
        if (threadIdx.x < kNaRow) {
            double s = 0.0;
            for (int ww = 0; ww < kNaThreads / 32; ww++) s += s_red[ww][threadIdx.x];
            a.scr->rows[(blockIdx.y * gridDim.x + blockIdx.x) * kNaRow + threadIdx.x] = s;
        }
    }
}

__global__ void k_na_finish(const NaArgs a, int n_rows) {
    const int k = threadIdx.x;
    if (k >= kNaRow) return;
    double s = 0.0;
    if (a.scr->bad) s = __longlong_as_double(0x7ff8000000000000ll);  // invalid input: NaN outputs
    else
        for (int r = 0; r < n_rows; r++) s += a.scr->rows[r * kNaRow + k];
    if (k == 0) {
        if (a.e) a.e[0] = s;
    } else if (k == 1) {
        if (a.e) a.e[1] = a.coul_fd * s;  // the Coulomb constant is applied once, in FP64
    } else if (a.vir) {
        a.vir[k - 2] = -0.25 * s;  // each pair was summed from both sides
    }
}

// device address of the scratch, looked up once per device (with that device
// current) and kept for the life of the process: after cudaDeviceReset the
// module is loaded again and this address is stale, so the entry point must not
// be used on a device after resetting it
std::mutex g_na_mutex;
NaScratch *g_na_addr[64] = {nullptr};

bool pos_finite(double v) { return isfinite(v) && v > 0.0; }

}  // namespace

extern "C" nb_status nb_forces_small_noalloc(const nb_params *p, const float *x_dev, const float *q_dev,
                                             const int32_t *type_dev, const int32_t *excl_off_dev,
                                             const int32_t *excl_idx_dev, const double *box_host, unsigned flags,
                                             float *f_dev, double *e_dev, double *vir_dev, void *stream) {
    // ---- host-side checks (no CUDA call before these pass)
    if (!p || !x_dev || !q_dev || !type_dev || !box_host || !f_dev || !p->c6_host || !p->c12_host)
        return NB_ERR_INVALID_ARG;
    if (flags & ~(unsigned)(NB_ENERGY | NB_VIRIAL)) return NB_ERR_INVALID_ARG;
    if ((flags & NB_ENERGY) && !e_dev) return NB_ERR_INVALID_ARG;
    if ((flags & NB_VIRIAL) && !vir_dev) return NB_ERR_INVALID_ARG;
    if ((excl_off_dev == nullptr) != (excl_idx_dev == nullptr)) return NB_ERR_INVALID_ARG;
    const int n = p->n_atoms, T = p->n_types;
    if (n < 1 || T < 1 || p->reserved != 0) return NB_ERR_INVALID_ARG;
    if (n > NB_NOALLOC_MAX_ATOMS || T > NB_NOALLOC_MAX_TYPES) return NB_ERR_CAPACITY;
    if (p->coulomb != NB_COULOMB_RF && p->coulomb != NB_COULOMB_EWALD && p->coulomb != NB_COULOMB_NONE)
        return NB_ERR_INVALID_ARG;
    if (!pos_finite(p->eps_r) || !pos_finite(p->rc) || isnan(p->eps_rf)) return NB_ERR_INVALID_ARG;
    if (p->coulomb == NB_COULOMB_EWALD && (!pos_finite(p->beta) || p->beta * p->rc > NB_EW_ZMAX_D))
        return NB_ERR_INVALID_ARG;
    for (int k = 0; k < 3; k++) {
        if (!pos_finite(box_host[k])) return NB_ERR_INVALID_ARG;
        if (!(p->rc < 0.5 * box_host[k])) return NB_ERR_BOX_TOO_SMALL;
    }
    for (int t = 0; t < T * T; t++)
        if (!isfinite(p->c6_host[t]) || !isfinite(p->c12_host[t])) return NB_ERR_INVALID_ARG;
    // ---- set-up: the scratch's device address, once per device
    int dev = 0;
    NB_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return NB_ERR_INVALID_ARG;
    NaScratch *scr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_addr[dev]) {
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_na_scratch);
            if (e != cudaSuccess) return nb_cuda_status(e);
            g_na_addr[dev] = static_cast<NaScratch *>(ptr);
        }
        scr = g_na_addr[dev];
    }
    // ---- arguments (tables by value: T <= NB_NOALLOC_MAX_TYPES)
    NaArgs a;
    memset(&a, 0, sizeof(a));
    const double rc = p->rc, rc3 = rc * rc * rc, rc6inv = 1.0 / (rc3 * rc3);
    a.v.rc2 = (float)(rc * rc);
    a.v.coul_f = (float)(138.935458 / p->eps_r);
    a.v.coul_f64 = 138.935458 / p->eps_r;
    const double krf = (!isfinite(p->eps_rf) || p->eps_rf <= 0.0)
                           ? 1.0 / (2.0 * rc3)
                           : (p->eps_rf - p->eps_r) / ((2.0 * p->eps_rf + p->eps_r) * rc3);
    const double crf = 1.0 / rc + krf * rc * rc;
    a.v.k_rf = (float)krf;
    a.v.c_rf = (float)crf;
    a.v.c_rf_lo = (float)(crf - (double)a.v.c_rf);
    a.v.ew_s = (float)(p->beta * p->beta / (NB_EW_ZMAX_D * NB_EW_ZMAX_D));
    a.v.ew_beta3 = (float)(p->beta * p->beta * p->beta);
    a.v.ew_beta = (float)p->beta;
    a.v.ew_shift = p->coulomb == NB_COULOMB_EWALD ? (float)(erfc(p->beta * rc) / rc) : 0.f;
    a.v.queue = nullptr;
    a.v.erow = nullptr;
    a.v.kept = nullptr;
    a.v.rin2 = 0.f;
    a.v.ew_beta2 = (float)(p->beta * p->beta);
    a.v.ew_beta_lo = (float)(p->beta - (double)a.v.ew_beta);
    a.v.ew_beta2_lo = (float)(p->beta * p->beta - (double)a.v.ew_beta2);
    a.v.ew_bt = a.v.ew_beta * (float)(1.0 / NB_EW_ZMAX_D);
    a.v.ew_bt_lo = a.v.ew_beta_lo * (float)(1.0 / NB_EW_ZMAX_D);
    a.v.ew_2bsp = (float)(2.0 * p->beta / sqrt(M_PI));
    a.v.rc6inv = (float)rc6inv;
    a.v.rc12inv = (float)(rc6inv * rc6inv);
    a.v.T = T;
    for (int x = 0; x < T; x++)
        for (int y = 0; y < T; y++) {
            const float s6 = 0.5f * (p->c6_host[x * T + y] + p->c6_host[y * T + x]);
            const float s12 = 0.5f * (p->c12_host[x * T + y] + p->c12_host[y * T + x]);
            a.lj[x * T + y] = make_float2(6.0f * s6, 12.0f * s12);
            const double sh = (double)s12 * rc6inv * rc6inv - (double)s6 * rc6inv;
            a.lje[x * T + y] = make_float4(s6, s12, (float)sh, 0.f);
        }
    a.n = n;
    a.T = T;
    for (int k = 0; k < 3; k++) {
        a.L[k] = box_host[k];
        a.Lhi[k] = (float)box_host[k];
        a.Llo[k] = (float)(box_host[k] - (double)a.Lhi[k]);
        a.half[k] = (float)(0.5 * box_host[k]);
    }
    a.coul_fd = 138.935458 / p->eps_r;
    a.x = x_dev;
    a.q = q_dev;
    a.type = type_dev;
    a.excl_off = excl_off_dev;
    a.excl_idx = excl_idx_dev;
    a.f = f_dev;
    a.e = (flags & NB_ENERGY) ? e_dev : nullptr;
    a.vir = (flags & NB_VIRIAL) ? vir_dev : nullptr;
    a.scr = scr;
    // ---- launches (the status word starts each call at zero)
    cudaStream_t st = (cudaStream_t)stream;
    const bool en = flags & (NB_ENERGY | NB_VIRIAL);
    const dim3 grid((n + kNaThreads - 1) / kNaThreads, kNaJSplit);
    NB_CUDA_TRY(cudaMemsetAsync(&scr->bad, 0, sizeof(int), st));
    k_na_prep<<<(n + 255) / 256, 256, 0, st>>>(a);
    if (p->coulomb == NB_COULOMB_RF) {
        if (en) k_na_forces<NB_COULOMB_RF, true><<<grid, kNaThreads, 0, st>>>(a);
        else k_na_forces<NB_COULOMB_RF, false><<<grid, kNaThreads, 0, st>>>(a);
    } else if (p->coulomb == NB_COULOMB_EWALD) {
        if (en) k_na_forces<NB_COULOMB_EWALD, true><<<grid, kNaThreads, 0, st>>>(a);
        else k_na_forces<NB_COULOMB_EWALD, false><<<grid, kNaThreads, 0, st>>>(a);
    } else {
        if (en) k_na_forces<NB_COULOMB_NONE, true><<<grid, kNaThreads, 0, st>>>(a);
        else k_na_forces<NB_COULOMB_NONE, false><<<grid, kNaThreads, 0, st>>>(a);
    }
    if (en) k_na_finish<<<1, 32, 0, st>>>(a, (int)(grid.x * grid.y));
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}
