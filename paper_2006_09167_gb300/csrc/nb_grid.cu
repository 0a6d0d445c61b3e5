// Grid sort and cluster bounding boxes (paper Sec. V.A and Fig. 4; Sec. V.D).
//
// Atoms are binned on a grid that is regular in x and y.  Each xy column is
// sorted by z and cut into super-cells of a fixed number of atoms (64), so the
// cells have a fixed atom count rather than a fixed size.  Each super-cell is
// split 2x2x2: by z into halves of 32, each half by y into quarters of 16, each
// quarter by x into the 8-atom clusters.  A column's last super-cell may be
// partial; its empty slots are padding (perm = -1) placed far outside the box
// at distinct positions so that no padding pair can fall inside any cut-off.
#include "nb_internal.cuh"

using namespace nbk;

namespace {

// ---------------------------------------------------------------- binning
__global__ void k_bin(int n, const float *__restrict__ x, double Lx, double Ly, double Lz,
                      double inv_cwx, double inv_cwy, int ncx, int ncy, int *__restrict__ col_count,
                      int *__restrict__ col_of, int *__restrict__ rank_of, float4 *__restrict__ wpos,
                      int *__restrict__ img, int *__restrict__ err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float xs[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    double L[3] = {Lx, Ly, Lz};
    float w[3];
    int im[3];
    for (int k = 0; k < 3; k++) {
        if (!isfinite(xs[k])) {
            record_error(err, NB_ERR_NONFINITE);
            xs[k] = 0.f;
        }
        double xd = (double)xs[k];
        double nd = floor(xd / L[k]);
        if (nd < -500.0 || nd > 500.0) {  // image offset field is 10 bits
            record_error(err, NB_ERR_INVALID_ARG);
            nd = 0.0;
        }
        double wd = xd - nd * L[k];
        float wf = (float)wd;
        if ((double)wf >= L[k]) {  // rounded onto L: use the next image (tiny negative coordinate)
            nd += 1.0;
            wf = (float)(xd - nd * L[k]);
        }
        if (nd == 0.0) wf = xs[k];  // exact for atoms already in the primary box
        w[k] = wf;
        im[k] = (int)nd;
    }
    int ix = (int)((double)w[0] * inv_cwx);
    int iy = (int)((double)w[1] * inv_cwy);
    ix = min(max(ix, 0), ncx - 1);
    iy = min(max(iy, 0), ncy - 1);
    int c = ix * ncy + iy;
    col_of[i] = c;
    rank_of[i] = atomicAdd(&col_count[c], 1);
    wpos[i] = make_float4(w[0], w[1], w[2], 0.f);
    img[i] = img_pack(im[0], im[1], im[2]);
}

// Exclusive scans over the columns (one block): atom offsets, super-cell offsets,
// the total super-cell count and the largest column.
__global__ void k_scan_cols(int ncol, const int *__restrict__ col_count, int *__restrict__ col_atom_off,
                            int *__restrict__ col_sc_off, int *__restrict__ counters) {
    __shared__ int s_a[1024], s_s[1024];
    __shared__ int carry_a, carry_s, s_max;
    if (threadIdx.x == 0) {
        carry_a = 0;
        carry_s = 0;
        s_max = 0;
    }
    __syncthreads();
    for (int base = 0; base < ncol; base += blockDim.x) {
        int c = base + threadIdx.x;
        int cnt = c < ncol ? col_count[c] : 0;
        if (cnt > 0) atomicMax(&s_max, cnt);
        s_a[threadIdx.x] = cnt;
        s_s[threadIdx.x] = (cnt + NB_SCA - 1) / NB_SCA;
        __syncthreads();
        for (int d = 1; d < blockDim.x; d <<= 1) {
            int va = threadIdx.x >= d ? s_a[threadIdx.x - d] : 0;
            int vs = threadIdx.x >= d ? s_s[threadIdx.x - d] : 0;
            __syncthreads();
            s_a[threadIdx.x] += va;
            s_s[threadIdx.x] += vs;
            __syncthreads();
        }
        if (c < ncol) {
            int incl_a = s_a[threadIdx.x], incl_s = s_s[threadIdx.x];
            col_atom_off[c] = carry_a + incl_a - cnt;
            col_sc_off[c] = carry_s + incl_s - (cnt + NB_SCA - 1) / NB_SCA;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) {
            carry_a += s_a[threadIdx.x];
            carry_s += s_s[threadIdx.x];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        col_atom_off[ncol] = carry_a;
        col_sc_off[ncol] = carry_s;
        counters[0] = carry_s;
        counters[1] = s_max;
    }
}

__global__ void k_scatter_cols(int n, const int *__restrict__ col_of, const int *__restrict__ rank_of,
                               const int *__restrict__ col_atom_off, int *__restrict__ colbuf) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    colbuf[col_atom_off[col_of[i]] + rank_of[i]] = i;
}

// One block per column: bitonic sort by (z, index), then stable rank sorts by
// (y, index) within 32-atom z-halves and by (x, index) within 16-atom quarters.
__global__ void k_sort_col(const int *__restrict__ col_count, const int *__restrict__ col_atom_off,
                           const int *__restrict__ col_sc_off, const int *__restrict__ colbuf,
                           const float4 *__restrict__ wpos, const float *__restrict__ q,
                           const int *__restrict__ type, int *__restrict__ perm, int *__restrict__ inv,
                           float4 *__restrict__ xq, int *__restrict__ type_s, float *__restrict__ q_s,
                           int *__restrict__ sc_col, int *__restrict__ err) {
    extern __shared__ unsigned long long sm[];
    const int c = blockIdx.x;
    const int n = col_count[c];
    if (n > NB_MAX_COL) {
        if (threadIdx.x == 0) record_error(err, NB_ERR_CAPACITY);
        return;
    }
    int P = 1;
    while (P < n) P <<= 1;
    unsigned long long *keys = sm;
    int *order = reinterpret_cast<int *>(sm + P);
    const int off = col_atom_off[c];
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        if (p < n) {
            int i = colbuf[off + p];
            keys[p] = ((unsigned long long)float_key(wpos[i].z) << 32) | (unsigned int)i;
        } else {
            keys[p] = ~0ull;
        }
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int p = threadIdx.x; p < P; p += blockDim.x) {
                int l = p ^ j;
                if (l > p) {
                    unsigned long long a = keys[p], b = keys[l];
                    bool up = (p & k) == 0;
                    if ((a > b) == up) {
                        keys[p] = b;
                        keys[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int p = threadIdx.x; p < n; p += blockDim.x) order[p] = (int)(keys[p] & 0xffffffffu);
    __syncthreads();
    // two stable rank passes: axis 1 (y) over segments of 32, axis 0 (x) over segments of 16
    for (int pass = 0; pass < 2; pass++) {
        const int seg = pass == 0 ? 32 : 16;
        int2 *pv = reinterpret_cast<int2 *>(keys);
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            int i = order[p];
            float4 w = wpos[i];
            pv[p] = make_int2(i, __float_as_int(pass == 0 ? w.y : w.x));
        }
        __syncthreads();
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            int s0 = p & ~(seg - 1);
            int s1 = min(s0 + seg, n);
            int2 me = pv[p];
            unsigned int mk = float_key(__int_as_float(me.y));
            int r = 0;
            for (int t = s0; t < s1; t++) {
                int2 o = pv[t];
                unsigned int ok = float_key(__int_as_float(o.y));
                r += (ok < mk) || (ok == mk && o.x < me.x);
            }
            order[s0 + r] = me.x;
        }
        __syncthreads();
    }
    const int sc0 = col_sc_off[c];
    const int nsc = col_sc_off[c + 1] - sc0;
    const int base = sc0 * NB_SCA;
    for (int p = threadIdx.x; p < nsc * NB_SCA; p += blockDim.x) {
        int slot = base + p;
        if (p < n) {
            int i = order[p];
            float4 w = wpos[i];
            float qi = q[i];
            perm[slot] = i;
            inv[i] = slot;
            xq[slot] = make_float4(w.x, w.y, w.z, qi);
            type_s[slot] = type[i];
            q_s[slot] = qi;
        } else {
            perm[slot] = -1;
            xq[slot] = pad_position(slot);
            type_s[slot] = 0;
            q_s[slot] = 0.f;
        }
    }
    for (int s = threadIdx.x; s < nsc; s += blockDim.x) sc_col[sc0 + s] = c;
}

// Cluster and super-cluster bounding boxes of the real atoms (padding ignored).
__global__ void k_bbox(int n_clusters, const int *__restrict__ perm, const float4 *__restrict__ xq,
                       float4 *__restrict__ bb, float4 *__restrict__ sbb) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    float lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f};
    if (c < n_clusters) {
        for (int a = 0; a < NB_CL; a++) {
            int s = c * NB_CL + a;
            if (perm[s] < 0) continue;
            float4 p = xq[s];
            lo[0] = fminf(lo[0], p.x);
            lo[1] = fminf(lo[1], p.y);
            lo[2] = fminf(lo[2], p.z);
            hi[0] = fmaxf(hi[0], p.x);
            hi[1] = fmaxf(hi[1], p.y);
            hi[2] = fmaxf(hi[2], p.z);
        }
        bb[2 * c] = make_float4(lo[0], lo[1], lo[2], 0.f);
        bb[2 * c + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
    for (int d = 1; d < NB_SCL; d <<= 1) {
        for (int k = 0; k < 3; k++) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], d));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], d));
        }
    }
    if (c < n_clusters && (c & (NB_SCL - 1)) == 0) {
        int si = c / NB_SCL;
        sbb[2 * si] = make_float4(lo[0], lo[1], lo[2], 0.f);
        sbb[2 * si + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
}

}  // namespace

// Phase 1 of the sort: bin, scan.  Returns after enqueueing; the caller reads
// counters[0..1] (super-cells, largest column) back before phase 2.
nb_status nb_launch_grid_sort_phase1(nb_ctx *c, const float *x, cudaStream_t st) {
    NB_CUDA_TRY(cudaMemsetAsync(c->col_count, 0, sizeof(int) * c->ncol, st));
    int nb = (c->N + 255) / 256;
    c->n_launches += 3;
    k_bin<<<nb, 256, 0, st>>>(c->N, x, c->box[0], c->box[1], c->box[2], 1.0 / c->cw[0], 1.0 / c->cw[1],
                              c->ncx, c->ncy, c->col_count, c->col_of, c->rank_of, c->wpos, c->img,
                              c->err);
    k_scan_cols<<<1, 1024, 0, st>>>(c->ncol, c->col_count, c->col_atom_off, c->col_sc_off, c->counters);
    k_scatter_cols<<<nb, 256, 0, st>>>(c->N, c->col_of, c->rank_of, c->col_atom_off, c->colbuf);
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}

nb_status nb_launch_grid_sort_phase2(nb_ctx *c, int max_col, cudaStream_t st) {
    int P = 1;
    while (P < max_col) P <<= 1;
    size_t smem = (size_t)P * (sizeof(unsigned long long) + sizeof(int));
    if (smem > 48 * 1024)
        NB_CUDA_TRY(cudaFuncSetAttribute(k_sort_col, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    int threads = P >= 1024 ? 1024 : (P >= 256 ? P : 256);
    c->n_launches += 2;
    k_sort_col<<<c->ncol, threads, smem, st>>>(c->col_count, c->col_atom_off, c->col_sc_off, c->colbuf,
                                               c->wpos, c->q, c->type, c->perm, c->inv, c->xq,
                                               c->type_s, c->q_s, c->sc_col, c->err);
    int ncl = c->S_host * NB_SCL;
    int nthr = ((ncl + 255) / 256) * 256;
    k_bbox<<<nthr / 256, 256, 0, st>>>(ncl, c->perm, c->xq, c->bb, c->sbb);
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}
