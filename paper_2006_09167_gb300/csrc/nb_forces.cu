// Cluster pair force kernel (paper Sec. V.A) and the per-step gather/scatter.
//
// One warp evaluates one work item: a super-cluster (8 i-clusters, 64 atoms),
// a periodic shift and a chunk of its joint j-list.  The loop order follows the
// paper: outer loop over j-clusters, inner loop over the 8 i-clusters, with
// whole cluster pairs skipped by the 8-bit interaction mask (a warp-uniform
// branch, so no divergence).  Lane (ti, tj) = (lane & 7, lane >> 3) computes
// the pairs (i-atom ti, j-atom tj) and (ti, tj + 4) of every 8x8 cluster pair,
// so each j-atom is loaded once per entry and reused for all 8 i-clusters.
// i-forces accumulate in per-warp shared memory for the whole item; j-forces are
// reduced over the 8 ti lanes by shuffles at the end of each j iteration and
// added once per j-atom.  Each pair is computed once (Newton's third law).  Exclusions and the
// self-pair triangle come from the entry's bit masks and are applied together
// with the cut-off test.  Pair arithmetic is FP32; energies and the virial are
// accumulated per lane in FP32 over one item and reduced in FP64.
//
// Separate kernels per Coulomb type and energy/virial output (template
// instantiations) avoid runtime conditionals in the inner loop (Sec. V.A).
//
// Ewald real space: force-only kernels use phi_C = f qi qj (1/r^3 - beta^3 H(z)),
// z = beta r, with the FMA-only rational H of ewald_rational.h; the energy
// kernels form exp(-z^2) once and take erfc(z) = exp(-z^2) X(z) and the force
// from it (nb_pair.cuh), V_C = f qi qj (erfc(z)/r - erfc(beta rc)/rc).
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "nb_pair.cuh"

using namespace nbk;

namespace {

// Warps (work items) per block, W: one where that keeps as many warps resident
// (few types: small tables per block), so that no warp waits at a block barrier
// for the others to run out of work; four where one-warp blocks would each hold a
// copy of large type-pair tables and fewer warps would fit an SM.
constexpr int kLj3MaxT = 8;  // largest type count with the T^3 parameter table (48 B x 512 = 24 KB)

// dynamic shared memory of the force kernel: the T x T tables, and for LJ3 the T^3 ones
__host__ __device__ inline size_t forces_smem(int T, bool en, bool lj3) {
    const size_t t2 = (size_t)T * T, t3 = lj3 ? t2 * T : 0;
    return t2 * (sizeof(float2) + (en ? sizeof(float4) : 0)) + t3 * (sizeof(float4) + (en ? sizeof(float4) + sizeof(float2) : 0));
}

// Persistent: a grid sized to the resident capacity of the GPU, each warp taking
// the next work item (ordered longest first) from a device counter, so the
// kernel tail is at most one item long (paper Sec. V.F: tails from uneven work).
template <int COUL, bool EN, bool VIR, bool PRUNE = false, bool LJ3 = false, int W = 4>
__global__ void __launch_bounds__(W * 32) k_forces(SysView v) {
    constexpr int kFW = W;
    extern __shared__ float4 s_dyn[];
    const int T = v.T, T2 = T * T, T3 = LJ3 ? T2 * T : 0;
    // float4 arrays first: lje [T2] (EN), l3f [T3], l3e [T3] (EN); then float2: lj [T2], l3s [T3] (EN)
    float4 *s_lje = s_dyn;
    float4 *s_l3f = s_lje + (EN ? T2 : 0);
    float4 *s_l3e = s_l3f + T3;
    float2 *s_lj = reinterpret_cast<float2 *>(s_l3e + (EN ? T3 : 0));
    float2 *s_l3s = s_lj + T2;
    __shared__ float4 s_xi[kFW][NB_SCA];
    __shared__ int s_ti[kFW][NB_SCA];
    __shared__ float s_fi[kFW][3 * NB_SCL * 32];
    for (int t = threadIdx.x; t < T2; t += blockDim.x) {
        s_lj[t] = v.lj[t];
        if (EN) s_lje[t] = v.lje[t];
    }
    if (LJ3) {
        // entry (a, b0, b1): the parameters of pairs (a, b0) and (a, b1), component-wise
        for (int t = threadIdx.x; t < T3; t += blockDim.x) {
            const int a = t / T2, b0 = (t / T) % T, b1 = t % T;
            const float2 f0 = v.lj[a * T + b0], f1 = v.lj[a * T + b1];
            s_l3f[t] = make_float4(f0.x, f1.x, f0.y, f1.y);
            if (EN) {
                const float4 e0 = v.lje[a * T + b0], e1 = v.lje[a * T + b1];
                s_l3e[t] = make_float4(e0.x, e1.x, e0.y, e1.y);
                s_l3s[t] = make_float2(e0.z, e1.z);
            }
        }
    }
    __syncthreads();
    const LjTables ljt = {s_lj, s_lje, s_l3f, s_l3e, s_l3s};
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned full = 0xffffffffu;
    // first item: the warp's index in the grid; later items from the counter,
    // which the gather zeroed (no burst of atomics at launch)
    const int n_warps = gridDim.x * kFW;
    int w = blockIdx.x * kFW + wib;
    double row = 0.0;  // lane < 11: FP64 sum of this warp's per-item partial sums
    while (w < v.n_items) {
        const int nj = PRUNE ? v.items[w].w : v.inner_len[w];
        KSum elj, ec;
        float vr[9];
#pragma unroll
        for (int k = 0; k < 9; k++) vr[k] = 0.f;
        if (nj > 0)
            process_item<COUL, EN, VIR, PRUNE, LJ3>(v, w, nj, ljt, s_xi[wib], s_ti[wib], s_fi[wib], elj, ec, vr);
        if (EN || VIR) {
            // FP32 warp reduction of the item's sums, added in FP64 to the warp's row
            warp_reduce_outputs<EN, VIR>(elj, ec, vr);
            if (lane < 11) {
                double val;
                if (lane == 0) val = (double)elj.s - (double)elj.c;
                else if (lane == 1) val = (double)ec.s - (double)ec.c;
                else val = (double)vr[lane - 2];
                row += val;
            }
        }
        __syncwarp();  // this warp's staging arrays are reused by its next item
        int claim = 0;
        if (lane == 0) claim = atomicAdd(v.queue, 1);
        w = n_warps + __shfl_sync(full, claim, 0);
    }
    // the block's rows of partial sums (one per warp), added in FP64 to slot (block mod
    // NB_EROW_SLOTS) of the context's block sums: the blocks spread their atomics over 32
    // addresses per value, so that they neither contend nor leave a backlog that would slow
    // the next kernel.  The last block to finish (a counter, no waiting) adds the slots and
    // writes the outputs (E_LJ, f E_C, -1/2 of the virial).
    if (EN || VIR) {
        __shared__ double s_row[kFW][11];
        __shared__ bool s_last;
        if (lane < 11) s_row[wib][lane] = row;
        __syncthreads();
        const int t = threadIdx.x;
        if (t < 11) {
            double tot = 0.0;
#pragma unroll
            for (int q = 0; q < kFW; q++) tot += s_row[q][t];
            atomicAdd(&v.erow[(blockIdx.x % NB_EROW_SLOTS) * 11 + t], tot);
            __threadfence();
        }
        __syncthreads();
        if (t == 0) s_last = atomicAdd(&v.queue[1], 1) == (int)gridDim.x - 1;
        __syncthreads();
        if (s_last && t < 11) {
            __threadfence();
            double tot = 0.0;
            for (int k = 0; k < NB_EROW_SLOTS; k++) tot += __ldcg(&v.erow[k * 11 + t]);
            if (t < 2) {
                if (v.e) v.e[t] = t == 0 ? tot : v.coul_f64 * tot;
            } else if (v.vir) {
                v.vir[t - 2] = -0.5 * tot;
            }
        }
    }
}

// Lines the force kernel will read from memory the gather does not write (inner
// list, item table, sorted types, exclusion masks): prefetched into L2 by the
// gather, so the force kernel's per-entry loads do not each wait for DRAM when
// the cache is cold.
struct L2Prefetch {
    const char *p[5];
    long long lines[5];  // 128-byte lines per region
};

// Positions of the step into the cluster layout (image offsets of the last sort),
// zeroing of the force accumulators and of the energy / virial outputs, and L2
// prefetch of the lists.
__global__ void k_gather(int nslots, const int *__restrict__ perm, const float *__restrict__ x,
                         const int *__restrict__ img, const float *__restrict__ q_s, double Lx, double Ly,
                         double Lz, float4 *__restrict__ xq, float4 *__restrict__ fs, double *e, double *vir,
                         int *err, int *queue, double *erow, L2Prefetch pf) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    for (int t = s; t < NB_EROW_SLOTS * 11; t += gridDim.x * blockDim.x) erow[t] = 0.0;
#pragma unroll
    for (int r = 0; r < 5; r++)
        if (s < pf.lines[r]) asm volatile("prefetch.global.L2 [%0];" ::"l"(pf.p[r] + (size_t)s * 128));
    if (s == 0) {
        queue[0] = queue[1] = 0;
        if (e) e[0] = e[1] = 0.0;
        if (vir)
            for (int k = 0; k < 9; k++) vir[k] = 0.0;
    }
    if (s >= nslots) return;
    fs[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int i = perm[s];
    if (i < 0) return;
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
    if (bad) record_error(err, NB_ERR_NONFINITE);
    xq[s] = make_float4(p[0], p[1], p[2], q_s[s]);
}

// Sorted-layout mode: zero the caller's sorted force array, the energy / virial
// outputs and the work-item counter, and prefetch the lists into L2 (as the
// gather does when it also brings in the positions).
__global__ void k_prep_sorted(int nslots, float4 *__restrict__ f, double *e, double *vir, int *queue, double *erow,
                              L2Prefetch pf) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    for (int t = s; t < NB_EROW_SLOTS * 11; t += gridDim.x * blockDim.x) erow[t] = 0.0;
#pragma unroll
    for (int r = 0; r < 5; r++)
        if (s < pf.lines[r]) asm volatile("prefetch.global.L2 [%0];" ::"l"(pf.p[r] + (size_t)s * 128));
    if (s == 0) {
        queue[0] = queue[1] = 0;
        if (e) e[0] = e[1] = 0.0;
        if (vir)
            for (int k = 0; k < 9; k++) vir[k] = 0.0;
    }
    if (s < nslots) f[s] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Forces back to caller order.
__global__ void k_unsort(int n, const int *__restrict__ inv, const float4 *__restrict__ fs, float *__restrict__ f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const float4 v = fs[inv[i]];
        f[3 * i] = v.x;
        f[3 * i + 1] = v.y;
        f[3 * i + 2] = v.z;
    }
}

// Resident blocks per SM of a force kernel variant (remembered per device and
// shared-memory size: the force call asks on every launch).
template <int COUL, bool EN, bool VIR, bool PRUNE, bool LJ3, int W>
int forces_occupancy(size_t smem) {
    static std::mutex mu;
    static std::vector<std::pair<size_t, int>> known;  // (smem * 64 + device, blocks)
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t key = smem * 64 + (size_t)(dev & 63);
    {
        std::lock_guard<std::mutex> lk(mu);
        for (const auto &k : known)
            if (k.first == key) return k.second;
    }
    if (smem > 16 * 1024)
        cudaFuncSetAttribute(k_forces<COUL, EN, VIR, PRUNE, LJ3, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_forces<COUL, EN, VIR, PRUNE, LJ3, W>, W * 32, smem) !=
            cudaSuccess ||
        occ < 1)
        occ = 1;
    std::lock_guard<std::mutex> lk(mu);
    if (known.size() < 64) known.emplace_back(key, occ);
    return occ;
}

// Returns the number of warps of the launch.
template <int COUL, bool EN, bool VIR, bool PRUNE = false, bool LJ3 = false, int W = 4>
int launch_forces_t(const SysView &v, int n_sm, cudaStream_t st) {
    constexpr int kFW = W;
    const size_t smem = forces_smem(v.T, EN, LJ3);
    // the type-pair tables of many types, with the 17 KB of static staging arrays,
    // exceed the default 48 KB of shared memory (64 types: 96 KB of tables); opt in
    // to the larger carve-out, at lower occupancy
    const int occ = forces_occupancy<COUL, EN, VIR, PRUNE, LJ3, W>(smem);
    const int blocks = std::min((v.n_items + kFW - 1) / kFW, std::max(n_sm, 1) * occ);
    k_forces<COUL, EN, VIR, PRUNE, LJ3, W><<<blocks, kFW * 32, smem, st>>>(v);
    return blocks * kFW;
}

// the T^3 parameter table where it fits (few types), the T x T tables otherwise; for
// the former, one-warp blocks where they keep as many warps resident as 4-warp ones
template <int COUL, bool EN, bool VIR>
int launch_pick(const SysView &v, int n_sm, cudaStream_t st) {
    if (v.T > kLj3MaxT) return launch_forces_t<COUL, EN, VIR, false, false, 4>(v, n_sm, st);
    const size_t smem = forces_smem(v.T, EN, true);
    const int warps1 = forces_occupancy<COUL, EN, VIR, false, true, 1>(smem);
    const int warps4 = 4 * forces_occupancy<COUL, EN, VIR, false, true, 4>(smem);
    return warps1 >= warps4 ? launch_forces_t<COUL, EN, VIR, false, true, 1>(v, n_sm, st)
                            : launch_forces_t<COUL, EN, VIR, false, true, 4>(v, n_sm, st);
}

}  // namespace

// Lines of the lists the force kernel reads, for an L2 prefetch before it runs.
static L2Prefetch list_prefetch(const nb_ctx *c, long long *most) {
    L2Prefetch pf;
    const int ns = c->S_host * NB_SCA;
    const bool lists = c->have_list;
    const void *base[5] = {c->cj_inner, c->items, c->inner_len, c->type_s, c->mask_lanes};
    const long long bytes[5] = {lists ? (long long)c->n_j * 8 : 0, lists ? (long long)c->n_items * 16 : 0,
                                lists ? (long long)c->n_items * 4 : 0, (long long)ns * 4,
                                lists ? (long long)c->n_masks * 64 : 0};
    *most = 0;
    for (int r = 0; r < 5; r++) {
        pf.p[r] = (const char *)base[r];
        pf.lines[r] = base[r] ? (bytes[r] + 127) / 128 : 0;
        *most = std::max(*most, pf.lines[r]);
    }
    return pf;
}

nb_status nb_launch_gather(nb_ctx *c, const float *x, double *e, double *vir, cudaStream_t st) {
    const int ns = c->S_host * NB_SCA;
    NbTraceScope tr(c, NB_TRACE_GATHER, st);
    c->n_launches++;
    c->xq_cur = nullptr;  // the positions of this call go to the context's own array
    long long most = 0;
    const L2Prefetch pf = list_prefetch(c, &most);
    const long long threads = std::max<long long>(ns, most);
    k_gather<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(ns, c->perm, x, c->img, c->q_s, c->box[0], c->box[1],
                                                                c->box[2], c->xq, c->fs, e, vir, c->err, c->queue,
                                                                c->erow, pf);
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}

// Returns the number of partial-sum rows written (one per warp of the launch).
int nb_dispatch_forces(const SysView &v, int coulomb, unsigned flags, int n_sm, cudaStream_t st) {
    const bool en = flags & NB_ENERGY, vi = flags & NB_VIRIAL;
    if (coulomb == NB_COULOMB_RF) {
        if (en && vi) return launch_pick<NB_COULOMB_RF, true, true>(v, n_sm, st);
        else if (en) return launch_pick<NB_COULOMB_RF, true, false>(v, n_sm, st);
        else if (vi) return launch_pick<NB_COULOMB_RF, false, true>(v, n_sm, st);
        else return launch_pick<NB_COULOMB_RF, false, false>(v, n_sm, st);
    } else if (coulomb == NB_COULOMB_EWALD) {
        if (en && vi) return launch_pick<NB_COULOMB_EWALD, true, true>(v, n_sm, st);
        else if (en) return launch_pick<NB_COULOMB_EWALD, true, false>(v, n_sm, st);
        else if (vi) return launch_pick<NB_COULOMB_EWALD, false, true>(v, n_sm, st);
        else return launch_pick<NB_COULOMB_EWALD, false, false>(v, n_sm, st);
    } else {
        if (en && vi) return launch_pick<NB_COULOMB_NONE, true, true>(v, n_sm, st);
        else if (en) return launch_pick<NB_COULOMB_NONE, true, false>(v, n_sm, st);
        else if (vi) return launch_pick<NB_COULOMB_NONE, false, true>(v, n_sm, st);
        else return launch_pick<NB_COULOMB_NONE, false, false>(v, n_sm, st);
    }
}


// Sorted-layout mode: prep (zeroing, prefetch), the force kernel on the caller's
// sorted positions and force array, and the fold of the energy / virial rows.
nb_status nb_launch_forces_sorted(nb_ctx *c, unsigned flags, const float4 *xq, float4 *f, double *e, double *vir,
                                  cudaStream_t st) {
    const int ns = c->S_host * NB_SCA;
    double *ee = (flags & NB_ENERGY) ? e : nullptr, *vv = (flags & NB_VIRIAL) ? vir : nullptr;
    long long most = 0;
    const L2Prefetch pf = list_prefetch(c, &most);
    const long long threads = std::max<long long>(ns, most);
    c->xq_cur = xq;  // the prune and the counts read this call's positions
    {
        NbTraceScope tr(c, NB_TRACE_GATHER, st);
        c->n_launches++;
        k_prep_sorted<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(ns, f, ee, vv, c->queue, c->erow, pf);
    }
    SysView v = nb_make_view(c, f, ee, vv);
    if (v.n_items > 0) {  // the force kernel also adds the energies and the virial to e and vir
        NbTraceScope tr(c, NB_TRACE_FORCES, st);
        nb_dispatch_forces(v, c->coulomb, flags, c->n_sm, st);
        c->n_launches++;
    }
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}

nb_status nb_launch_forces(nb_ctx *c, unsigned flags, float *f, double *e, double *vir, cudaStream_t st,
                           bool fused_prune) {
    SysView v = nb_make_view(c, c->fs, (flags & NB_ENERGY) ? e : nullptr, (flags & NB_VIRIAL) ? vir : nullptr);
    if (v.n_items > 0) {  // the force kernel also adds the energies and the virial to e and vir
        NbTraceScope tr(c, NB_TRACE_FORCES, st);
        if (fused_prune) {
            // first use of a new list: the outer list, pruned on the way (energies and the
            // virial are always formed; they are added to e and vir only if requested)
            v.cj = c->cj_outer;
            v.kept = c->kept;
            const float re = (float)c->r_in * (1.0f + 2e-6f);  // as the separate prune pass
            v.rin2 = re * re;
            if (c->coulomb == NB_COULOMB_RF) launch_forces_t<NB_COULOMB_RF, true, true, true>(v, c->n_sm, st);
            else if (c->coulomb == NB_COULOMB_EWALD) launch_forces_t<NB_COULOMB_EWALD, true, true, true>(v, c->n_sm, st);
            else launch_forces_t<NB_COULOMB_NONE, true, true, true>(v, c->n_sm, st);
        } else {
            nb_dispatch_forces(v, c->coulomb, flags, c->n_sm, st);
        }
        c->n_launches++;
    }
    const int nb = (c->N + 255) / 256;
    c->n_launches++;
    k_unsort<<<nb, 256, 0, st>>>(c->N, c->inv, c->fs, f);
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}
