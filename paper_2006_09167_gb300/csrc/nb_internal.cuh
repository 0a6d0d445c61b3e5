// Internal definitions shared by the CUDA translation units of libnb.
// Layout (all in device memory, sorted "cluster" order):
//   slot s = 64*si + 8*k + a : atom a of cluster k of super-cluster si
//   xq[s]   float4 (x, y, z, q)  positions at the last gather (image fixed at grid sort)
//   perm[s] caller index of the atom in slot s, -1 for a padding slot
// Pair lists:
//   item  int4 {si, shift index, j_start, outer length}; inner length in inner_len[item]
//   outer entry int2 {cj, meta}: meta bits 0..7 interaction mask (bit k: i-cluster k of si),
//         bits 8..31 = 1 + index of a group of 8 uint64 exclusion masks (0: none)
//   inner entry int2: the prune keeps one bit per (i-cluster, j-half) (j-cluster splitting):
//         x = cj | hi << 24, y = lo | (exclusion group + 1) << 8, where bit k of lo (hi) says
//         that i-cluster k interacts with j-atoms 0..3 (4..7) of cj
//   exclusion mask u64 per (i-cluster k, j-cluster): bit 8*a + b set = pair (i-atom a,
//         j-atom b) interacts (cleared for excluded pairs, the lower triangle and padding
//         of a self cluster pair).
//   mask_lanes u16 [group][32 lanes]: the same bits in the pair kernels' lane order: lane
//         (ti, tj) = (lane & 7, lane >> 3) holds at bit 2k + h the bit of pair (i-atom ti,
//         j-atom tj + 4h) of i-cluster k.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/nb.h"

#define NB_CL 8            // atoms per cluster
#define NB_SCL 8           // clusters per super-cluster (2x2x2)
#define NB_SCA 64          // atoms per super-cluster
#define NB_MAX_EXCL 16     // exclusion partners per atom
#define NB_EROW_SLOTS 32   // addresses the force kernel's blocks spread their energy / virial sums over
#define NB_LJ3_MAX_T 8     // types up to which the T^3 parameter tables are kept (48 B x 512)
#define NB_MAX_COL 8192    // atoms per grid column (bitonic sort in shared memory)
#define NB_MAX_TYPES 64
#define NB_PAD_COORD -1.0e5f
#define NB_PAD_STEP 16.0f  // z spacing of padding positions between clusters
#define NB_SHIFT_CENTER 13 // shift index of (0,0,0); index = 9*(sx+1) + 3*(sy+1) + (sz+1)
#define NB_EW_ZMAX_D 4.0   // beta*rc limit of the Ewald rational approximations

namespace nbk {

struct Item {
    int si, shift, j_start, len;
};

// Per-system view used by the pair kernels (also one per replica in the batched kernel).
struct SysView {
    const float4 *xq;
    const int *type;
    const int4 *items;
    const int *inner_len;
    const int2 *cj;
    const unsigned long long *masks;
    const unsigned short *mask_lanes;
    const float2 *lj;   // [T*T] (6*C6, 12*C12), symmetrised
    const float4 *lje;  // [T*T] (C6, C12, C12/rc^12 - C6/rc^6, 0), symmetrised
    const float4 *l3f, *l3e;  // [T^3] or nullptr: (6 C6, 6 C6', 12 C12, 12 C12'), (C6, C6', C12, C12')
    const float2 *l3s;        // [T^3] or nullptr: (shift, shift')
    float4 *f;          // sorted force accumulators
    double *e;          // [2] or nullptr
    double *vir;        // [9] or nullptr
    int n_items;
    int T;
    float box_hi[3], box_lo[3];  // L as float plus the float remainder L - (float)L
    float rc2;
    float coul_f;  // 138.935458 / eps_r
    double coul_f64;  // the same in FP64 (applied to the Coulomb energy sum)
    float k_rf, c_rf, c_rf_lo;  // c_rf as a float pair (c_rf + c_rf_lo)
    float ew_s;      // beta^2 / ZMAX^2
    float ew_beta3;  // beta^3
    float ew_beta;   // beta (float pair with ew_beta_lo)
    float ew_shift;  // erfc(beta rc)/rc (without the Coulomb constant)
    float ew_beta2;  // beta^2 (float pair with ew_beta2_lo)
    float ew_beta_lo, ew_beta2_lo;  // beta - (float)beta, beta^2 - (float)beta^2
    float ew_2bsp;   // 2 beta / sqrt(pi)
    float ew_bt, ew_bt_lo;  // beta / ZMAX as a float pair (X(z) is evaluated in t = z / ZMAX)
    float rc6inv, rc12inv;
    int *queue;  // [0] work-item counter of the persistent force kernel, [1] its finished blocks (zeroed by the gather)
    double *erow;  // [NB_EROW_SLOTS * 11] energy / virial sums of the force kernel's blocks, by slot (zeroed by the gather)
    unsigned short *kept;  // first-use prune fused into the force kernel: half masks per outer entry
    float rin2;            // and its squared inner radius
};

// inner-entry decoding
__host__ __device__ __forceinline__ int inner_cj(int2 e) { return e.x & 0xffffff; }
__host__ __device__ __forceinline__ int inner_lo(int2 e) { return e.y & 0xff; }
__host__ __device__ __forceinline__ int inner_hi(int2 e) { return (int)((unsigned)e.x >> 24); }
__host__ __device__ __forceinline__ int entry_group(int2 e) { return (int)((unsigned)e.y >> 8); }

__device__ __forceinline__ void record_error(int *flag, int code) {
    if (flag) atomicCAS(flag, 0, code);
}

__host__ __device__ __forceinline__ void shift_of(int sidx, int &sx, int &sy, int &sz) {
    sx = sidx / 9 - 1;
    sy = (sidx / 3) % 3 - 1;
    sz = sidx % 3 - 1;
}

__host__ __device__ __forceinline__ float4 pad_position(int slot) {
    return make_float4(NB_PAD_COORD, NB_PAD_COORD, NB_PAD_COORD - NB_PAD_STEP * (float)(slot >> 3), 0.f);
}

// One Newton step for y ~ 1/sqrt(x) written on the residual e = 1 - x y^2
// (formed with an FMA) so that the update y + y e / 2 is a small increment:
// the result is within about one ulp and, unlike y (1.5 - x y^2 / 2) evaluated
// in FP32, carries no rounding bias.  Energies sum millions of r^-12 terms, so a
// bias of a fraction of an ulp in 1/r would show up in the total.
__device__ __forceinline__ float rsqrt_refine(float x, float y) {
    const float e = fmaf(-(x * y), y, 1.0f);
    return fmaf(0.5f * y, e, y);
}

// order-preserving map of a float to uint32 (handles negative values)
__device__ __forceinline__ unsigned int float_key(float v) {
    unsigned int u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// packed periodic image offsets (10 bits per axis, biased by 512)
__host__ __device__ __forceinline__ int img_pack(int nx, int ny, int nz) {
    return ((nx + 512) & 1023) | (((ny + 512) & 1023) << 10) | (((nz + 512) & 1023) << 20);
}
__host__ __device__ __forceinline__ void img_unpack(int p, int &nx, int &ny, int &nz) {
    nx = (p & 1023) - 512;
    ny = ((p >> 10) & 1023) - 512;
    nz = ((p >> 20) & 1023) - 512;
}

}  // namespace nbk

struct nb_ctx {
    // problem
    int N = 0, T = 0, coulomb = 0;
    double eps_r = 1, eps_rf = 0, beta = 0, rc = 0, rlist = 0, r_in = 0;
    int excl_n = 0;
    // device inputs (caller order)
    float *q = nullptr;
    int *type = nullptr;
    int *excl_off = nullptr, *excl_idx = nullptr;
    float2 *lj = nullptr;
    float4 *lje = nullptr;
    // for at most NB_LJ3_MAX_T types: the same parameters by (i-type, j-type, j-type'),
    // both pairs of a packed iteration in one entry (read by the batched kernel)
    float4 *l3f = nullptr, *l3e = nullptr;
    float2 *l3s = nullptr;
    // grid
    bool have_grid = false;
    double box[3] = {0, 0, 0};
    int ncx = 0, ncy = 0, ncol = 0, ncol_cap = 0;
    double cw[2] = {0, 0};
    int S_cap = 0;  // super-cluster capacity (upper bound on the count after a sort)
    int *col_count = nullptr, *col_atom_off = nullptr, *col_sc_off = nullptr;
    int *counters = nullptr;  // [16] device scalars (0: S, 1: max column count, ...)
    int *col_of = nullptr, *rank_of = nullptr, *colbuf = nullptr, *img = nullptr;
    float4 *wpos = nullptr;
    int N_cap = 0;
    // sorted layout
    float4 *xq = nullptr;
    const float4 *xq_cur = nullptr;  // positions of the last force call: xq, or the caller's (sorted mode)
    int *type_s = nullptr, *perm = nullptr, *inv = nullptr, *sc_col = nullptr;
    float *q_s = nullptr;
    float4 *bb = nullptr;   // [S_cap*8*2]
    float4 *sbb = nullptr;  // [S_cap*2]
    float4 *fs = nullptr;   // [S_cap*64]
    float4 *gfs = nullptr, *gxs = nullptr;  // adjoint: sorted gF, dL/dx  [S_cap*64]
    float *gqs = nullptr;                   // adjoint: sorted dL/dq      [S_cap*64]
    double *gpar = nullptr;                 // adjoint: [2*T*T] parameter gradients
    int S_host = 0;         // exact super-cluster count (read back by the list build)
    // lists
    bool have_list = false;
    float rlist_built = 0.f;
    bool fused_prune = false;    // first prune after a build inside the first force call
    bool inner_pending = false;  // the inner list awaits that first prune
    int split = 16;          // max outer j-entries per work item (next build)
    int search_seg = 0;      // column segments of the pair search (0: the library's choice; next build)
    int split_built = 16;    // max outer j-entries per work item of the current lists
    int n_items = 0, n_j = 0, n_masks = 0;
    int items_cap = 0, j_cap = 0, masks_cap = 0, si_cap = 0;
    int4 *items = nullptr, *items_tmp = nullptr;
    int *inner_len = nullptr;
    int2 *cj_outer = nullptr, *cj_inner = nullptr, *cj_tmp = nullptr;
    unsigned long long *masks = nullptr;
    unsigned short *mask_lanes = nullptr;  // [32 * masks_cap] the masks in lane order
    int *si_counts = nullptr;  // [4*si_cap]: j entries, items, mask groups, bits per search unit
    int *si_offs = nullptr;    // [4*(si_cap+1)]
    int *sort_tmp = nullptr;   // item sort scratch
    unsigned short *kept = nullptr;  // [j_cap] prune scratch: surviving half masks per outer entry
    int sort_tmp_cap = 0;
    int64_t n_outer_bits = 0;
    // diagnostics
    long long *diag = nullptr;  // [4]
    int *err = nullptr;
    int *queue = nullptr;  // [2] work-item counter and finished-block counter of the persistent force kernel
    double *erow = nullptr;  // [NB_EROW_SLOTS * 11] block sums of energies and virial
    double *ewald_part = nullptr;    // [1024*8] per-block rows of the Ewald exclusion / self kernel
    unsigned *ewald_count = nullptr;  // its finished-block counter (zero between calls)
    int n_sm = 0;          // multiprocessors of the context's device
    long long n_launches = 0;
    // tracing: event pairs per traced kernel kind
    unsigned trace_mask = 0;  // bit k: launches of trace kind k are timed
    std::vector<cudaEvent_t> ev_start[NB_TRACE_KINDS], ev_end[NB_TRACE_KINDS];
    int ev_used[NB_TRACE_KINDS] = {0, 0, 0, 0};
};

// Record the start / end of a traced kernel (no-ops when tracing is off or full).
struct NbTraceScope {
    nb_ctx *c;
    int kind;
    cudaStream_t st;
    bool on;
    NbTraceScope(nb_ctx *c_, int kind_, cudaStream_t st_) : c(c_), kind(kind_), st(st_) {
        on = ((c->trace_mask >> kind) & 1u) && c->ev_used[kind] < (int)c->ev_start[kind].size();
        if (on) cudaEventRecord(c->ev_start[kind][c->ev_used[kind]], st);
    }
    ~NbTraceScope() {
        if (on) {
            cudaEventRecord(c->ev_end[kind][c->ev_used[kind]], st);
            c->ev_used[kind]++;
        }
    }
};

// helpers implemented in nb_api.cu
nb_status nb_cuda_status(cudaError_t e);
#define NB_CUDA_TRY(call)                                \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return nb_cuda_status(_e); \
    } while (0)

nbk::SysView nb_make_view(const nb_ctx *c, float4 *f, double *e, double *vir);
// positions of the last force call (sorted mode: the caller's array), else of the last gather or sort
inline const float4 *nb_cur_xq(const nb_ctx *c) { return c->xq_cur ? c->xq_cur : c->xq; }

// launchers (one per translation unit)
nb_status nb_launch_grid_sort(nb_ctx *c, const float *x, cudaStream_t st);
nb_status nb_launch_search(nb_ctx *c, float rlist, cudaStream_t st);
nb_status nb_launch_prune(nb_ctx *c, float r_in, int part, int n_parts, cudaStream_t st);
nb_status nb_launch_gather(nb_ctx *c, const float *x, double *e, double *vir, cudaStream_t st);
nb_status nb_launch_prune_compact_all(nb_ctx *c, cudaStream_t st);
nb_status nb_ensure_inner(nb_ctx *c, cudaStream_t st);
nb_status nb_launch_forces(nb_ctx *c, unsigned flags, float *f, double *e, double *vir,
                           cudaStream_t st, bool fused_prune = false);
nb_status nb_launch_forces_sorted(nb_ctx *c, unsigned flags, const float4 *xq, float4 *f, double *e, double *vir,
                                  cudaStream_t st);
nb_status nb_launch_count(nb_ctx *c, int which, cudaStream_t st);
nb_status nb_launch_export(nb_ctx *c, int which, long long *buf, long long cap, long long *count,
                           cudaStream_t st);
nb_status nb_launch_vjp(nb_ctx *c, const float *x, const float *gF, double gE, const double *gE_dev, float *gx,
                        float *gq, double *gc6, double *gc12, cudaStream_t st);
