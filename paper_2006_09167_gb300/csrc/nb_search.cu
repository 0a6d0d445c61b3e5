// Bounding-box cluster pair search (paper Sec. V.A, Fig. 4 right; Sec. V.D).
//
// For every super-cluster si (8 i-clusters) and periodic shift s, the joint
// j-list is the union of j-clusters whose bounding box lies within rlist of
// the (shifted) bounding box of any of the 8 i-clusters; the 8-bit interaction
// mask of each entry says which i-clusters are in range.  Each cluster pair is
// listed once (Newton's third law): (ci, cj, s) with cj > ci for any shift, or
// cj == ci with shift index >= the centre (s = 0 is the self pair, evaluated
// with an upper-triangle mask).  Exclusions are stored with the j-cluster
// entries as 8x8 bit masks.  Lists are cut into work items of at most `split`
// entries and the items are ordered longest first (Sec. V.F).
//
// The search runs twice: a counting pass sizes every super-cluster's output,
// an exclusive scan turns the counts into offsets, and a writing pass emits
// entries in a fixed order, so the list is deterministic.  Each super-cluster's
// grid columns are split into `seg` segments (1 to 8; column index mod seg), each
// a search unit with its own count and offset searched by one warp, and work
// items hold the entries of one shift and one segment.
#include "nb_internal.cuh"

using namespace nbk;

namespace {

constexpr int kWarps = 4;
constexpr int kSegMax = 8;          // most warps (column segments) per super-cluster
constexpr int kSegWarps = 12000;    // segments are doubled while the search has fewer warps than this

struct SearchArgs {
    int S;
    const float4 *bb, *sbb;
    const int *col_sc_off;
    int ncx, ncy;
    float cwx, cwy;
    float L[3];
    float rlist, rlist2;
    const int *perm, *inv, *excl_off, *excl_idx;
    int split;
    int seg;             // column segments (one warp each) per super-cluster
    int *si_counts;      // count pass: [4*S] j entries, items, mask groups, mask bits
    const int *si_offs;  // write pass: [4*(S+1)] exclusive offsets
    int4 *items;
    int2 *cj_out;
    unsigned long long *masks;
};

__device__ __forceinline__ float box_d2(float4 alo, float4 ahi, float4 blo, float4 bhi) {
    float dx = fmaxf(0.f, fmaxf(blo.x - ahi.x, alo.x - bhi.x));
    float dy = fmaxf(0.f, fmaxf(blo.y - ahi.y, alo.y - bhi.y));
    float dz = fmaxf(0.f, fmaxf(blo.z - ahi.z, alo.z - bhi.z));
    return dx * dx + dy * dy + dz * dz;
}

template <bool WRITE>
__global__ void __launch_bounds__(kWarps * 32) k_search(SearchArgs a) {
    __shared__ int s_part[kWarps][NB_SCA][NB_MAX_EXCL];
    __shared__ int s_pcnt[kWarps][NB_SCA];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int unit = blockIdx.x * kWarps + wib;  // (super-cluster, column segment)
    const int si = unit / a.seg, seg = unit % a.seg;
    if (si >= a.S) return;
    const unsigned full = 0xffffffffu;

    // exclusion partners (as sorted slots) of the 64 i-atoms
    for (int h = 0; h < 2; h++) {
        int at = lane + 32 * h;
        int i = a.perm[si * NB_SCA + at];
        int cnt = 0;
        if (i >= 0) {
            for (int e = a.excl_off[i]; e < a.excl_off[i + 1] && cnt < NB_MAX_EXCL; e++)
                s_part[wib][at][cnt++] = a.inv[a.excl_idx[e]];
        }
        s_pcnt[wib][at] = cnt;
    }
    __syncwarp();

    const int k0 = (lane & 3) * 2, k1 = k0 + 1, jc = lane >> 2;
    const float4 ilo0 = a.bb[2 * (si * NB_SCL + k0)], ihi0 = a.bb[2 * (si * NB_SCL + k0) + 1];
    const float4 ilo1 = a.bb[2 * (si * NB_SCL + k1)], ihi1 = a.bb[2 * (si * NB_SCL + k1) + 1];
    const bool ie0 = ilo0.x > ihi0.x, ie1 = ilo1.x > ihi1.x;
    const float4 slo = a.sbb[2 * si], shi = a.sbb[2 * si + 1];
    const int row_base = si * NB_SCA;
    // pad flags of the 64 i-slots, used for self masks
    const unsigned long long padbits =
        ((unsigned long long)__ballot_sync(full, a.perm[row_base + 32 + lane] < 0) << 32) |
        (unsigned long long)__ballot_sync(full, a.perm[row_base + lane] < 0);

    int n_j = 0, n_items = 0, n_masks = 0, n_bits = 0;
    int j_base = 0, it_base = 0, m_base = 0;
    if (WRITE) {
        j_base = a.si_offs[4 * unit + 0];
        it_base = a.si_offs[4 * unit + 1];
        m_base = a.si_offs[4 * unit + 2];
    }

    for (int sidx = 0; sidx < 27; sidx++) {
        int sh[3];
        shift_of(sidx, sh[0], sh[1], sh[2]);
        const float slo_a[3] = {slo.x, slo.y, slo.z}, shi_a[3] = {shi.x, shi.y, shi.z};
        bool ok = true;
        for (int k = 0; k < 3; k++) {
            if (sh[k] == 1 && !(slo_a[k] < a.rlist)) ok = false;
            if (sh[k] == -1 && !(a.L[k] - shi_a[k] < a.rlist)) ok = false;
        }
        if (!ok) continue;
        const float3 sv = make_float3(sh[0] * a.L[0], sh[1] * a.L[1], sh[2] * a.L[2]);
        const float4 tlo = make_float4(slo.x + sv.x, slo.y + sv.y, slo.z + sv.z, 0.f);
        const float4 thi = make_float4(shi.x + sv.x, shi.y + sv.y, shi.z + sv.z, 0.f);
        const float4 clo0 = make_float4(ilo0.x + sv.x, ilo0.y + sv.y, ilo0.z + sv.z, 0.f);
        const float4 chi0 = make_float4(ihi0.x + sv.x, ihi0.y + sv.y, ihi0.z + sv.z, 0.f);
        const float4 clo1 = make_float4(ilo1.x + sv.x, ilo1.y + sv.y, ilo1.z + sv.z, 0.f);
        const float4 chi1 = make_float4(ihi1.x + sv.x, ihi1.y + sv.y, ihi1.z + sv.z, 0.f);
        int ix0 = (int)floorf((tlo.x - a.rlist) / a.cwx), ix1 = (int)floorf((thi.x + a.rlist) / a.cwx);
        int iy0 = (int)floorf((tlo.y - a.rlist) / a.cwy), iy1 = (int)floorf((thi.y + a.rlist) / a.cwy);
        ix0 = max(ix0, 0);
        iy0 = max(iy0, 0);
        ix1 = min(ix1, a.ncx - 1);
        iy1 = min(iy1, a.ncy - 1);
        int cur_len = 0;  // entries in the open item of this shift
        int cur_start = n_j;
        for (int ix = ix0; ix <= ix1; ix++) {
            for (int iy = iy0; iy <= iy1; iy++) {
                const int col = ix * a.ncy + iy;
                if (col % a.seg != seg) continue;
                const int sa = max(a.col_sc_off[col], si), sb = a.col_sc_off[col + 1];
                for (int c0 = sa; c0 < sb; c0 += 32) {
                    const int sj = c0 + lane;
                    bool cand = false;
                    if (sj < sb) {
                        float4 jlo = a.sbb[2 * sj], jhi = a.sbb[2 * sj + 1];
                        cand = jlo.x <= jhi.x && box_d2(tlo, thi, jlo, jhi) < a.rlist2;
                    }
                    unsigned cm = __ballot_sync(full, cand);
                    while (cm) {
                        const int sjj = c0 + __ffs(cm) - 1;
                        cm &= cm - 1;
                        const int cj = sjj * NB_SCL + jc;
                        const float4 jlo = a.bb[2 * cj], jhi = a.bb[2 * cj + 1];
                        const bool je = jlo.x > jhi.x;
                        const int ci0 = si * NB_SCL + k0, ci1 = ci0 + 1;
                        bool t0 = !ie0 && !je && (cj > ci0 || (cj == ci0 && sidx >= NB_SHIFT_CENTER)) &&
                                  box_d2(clo0, chi0, jlo, jhi) < a.rlist2;
                        bool t1 = !ie1 && !je && (cj > ci1 || (cj == ci1 && sidx >= NB_SHIFT_CENTER)) &&
                                  box_d2(clo1, chi1, jlo, jhi) < a.rlist2;
                        int bits = ((int)t0 << k0) | ((int)t1 << k1);
                        bits |= __shfl_xor_sync(full, bits, 1);
                        bits |= __shfl_xor_sync(full, bits, 2);
                        unsigned em = __ballot_sync(full, (lane & 3) == 0 && bits != 0);
                        while (em) {
                            const int src = __ffs(em) - 1;
                            em &= em - 1;
                            const int imask = __shfl_sync(full, bits, src);
                            const int ecj = sjj * NB_SCL + (src >> 2);
                            // exclusion bits of this (super-cluster, j-cluster) pair
                            unsigned long long ex[2];
                            for (int h = 0; h < 2; h++) {
                                const int at = lane + 32 * h;
                                unsigned row = 0;
                                const int pc = s_pcnt[wib][at];
                                for (int e = 0; e < pc; e++) {
                                    int ps = s_part[wib][at][e];
                                    if ((ps >> 3) == ecj) row |= 1u << (ps & 7);
                                }
                                unsigned long long v = (unsigned long long)row << (8 * (lane & 7));
                                v |= __shfl_xor_sync(full, v, 1);
                                v |= __shfl_xor_sync(full, v, 2);
                                v |= __shfl_xor_sync(full, v, 4);
                                ex[h] = v;  // lanes 8g..8g+7 hold cluster g (h=0) or 4+g (h=1)
                            }
                            const bool any_ex = __any_sync(full, (ex[0] | ex[1]) != 0ull);
                            const bool self = (sjj == si) && (sidx == NB_SHIFT_CENTER);
                            const bool has = any_ex || self;
                            if (WRITE) {
                                int meta = imask;
                                if (has) {
                                    const int g = m_base + n_masks;
                                    meta |= (g + 1) << 8;
                                    // lane 8g writes cluster g and 4+g
                                    if ((lane & 7) == 0) {
                                        const int kk[2] = {lane >> 3, 4 + (lane >> 3)};
                                        for (int h = 0; h < 2; h++) {
                                            unsigned long long m = ~ex[h];
                                            if (self && kk[h] == (src >> 2)) {
                                                unsigned long long tri = 0ull;
                                                unsigned long long pad =
                                                    (padbits >> (8 * kk[h])) & 0xffull;
                                                for (int ia = 0; ia < 8; ia++)
                                                    for (int jb = ia + 1; jb < 8; jb++)
                                                        if (!((pad >> ia) & 1) && !((pad >> jb) & 1))
                                                            tri |= 1ull << (8 * ia + jb);
                                                m &= tri;
                                            }
                                            a.masks[(size_t)g * 8 + kk[h]] = m;
                                        }
                                    }
                                }
                                if (lane == 0) a.cj_out[j_base + n_j] = make_int2(ecj, meta);
                            }
                            if (has) n_masks++;
                            n_bits += __popc(imask);
                            n_j++;
                            cur_len++;
                            if (cur_len == a.split) {
                                if (WRITE && lane == 0)
                                    a.items[it_base + n_items] =
                                        make_int4(si, sidx, j_base + cur_start, cur_len);
                                n_items++;
                                cur_len = 0;
                                cur_start = n_j;
                            }
                        }
                    }
                }
            }
        }
        if (cur_len > 0) {
            if (WRITE && lane == 0)
                a.items[it_base + n_items] = make_int4(si, sidx, j_base + cur_start, cur_len);
            n_items++;
        }
    }
    if (!WRITE && lane == 0) {
        a.si_counts[4 * unit + 0] = n_j;
        a.si_counts[4 * unit + 1] = n_items;
        a.si_counts[4 * unit + 2] = n_masks;
        a.si_counts[4 * unit + 3] = n_bits;
    }
}

// Exclusive scan of 4 interleaved int streams of length n (one block of 1024 threads);
// offs[4*n..4*n+3] = totals.  Thread t sums a contiguous run of the units, a
// shuffle scan over the block turns the run sums into run offsets, and each thread
// then writes its run's offsets.
__global__ void k_scan4(int n, const int *__restrict__ cnt, int *__restrict__ offs) {
    __shared__ int4 s_warp[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b = min(n, t * per), e = min(n, b + per);
    const int4 *c4 = reinterpret_cast<const int4 *>(cnt);
    int4 sum = make_int4(0, 0, 0, 0);
#pragma unroll 8
    for (int i = b; i < e; i++) {
        const int4 v = c4[i];
        sum = make_int4(sum.x + v.x, sum.y + v.y, sum.z + v.z, sum.w + v.w);
    }
    // inclusive scan of the run sums within the warp, then over the warps
    int4 inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, inc.x, o), y = __shfl_up_sync(0xffffffffu, inc.y, o);
        const int z = __shfl_up_sync(0xffffffffu, inc.z, o), w = __shfl_up_sync(0xffffffffu, inc.w, o);
        if (lane >= o) inc = make_int4(inc.x + x, inc.y + y, inc.z + z, inc.w + w);
    }
    if (lane == 31) s_warp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int4 v = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : make_int4(0, 0, 0, 0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, v.x, o), y = __shfl_up_sync(0xffffffffu, v.y, o);
            const int z = __shfl_up_sync(0xffffffffu, v.z, o), w = __shfl_up_sync(0xffffffffu, v.w, o);
            if (lane >= o) v = make_int4(v.x + x, v.y + y, v.z + z, v.w + w);
        }
        s_warp[lane] = v;  // inclusive over warps
    }
    __syncthreads();
    const int4 wbase = wid > 0 ? s_warp[wid - 1] : make_int4(0, 0, 0, 0);
    int4 run = make_int4(wbase.x + inc.x - sum.x, wbase.y + inc.y - sum.y, wbase.z + inc.z - sum.z,
                         wbase.w + inc.w - sum.w);
    int4 *o4 = reinterpret_cast<int4 *>(offs);
#pragma unroll 8
    for (int i = b; i < e; i++) {
        o4[i] = run;
        const int4 v = c4[i];
        run = make_int4(run.x + v.x, run.y + v.y, run.z + v.z, run.w + v.w);
    }
    if (t == blockDim.x - 1) {
        const int4 tot = s_warp[(blockDim.x >> 5) - 1];
        offs[4 * n] = tot.x;
        offs[4 * n + 1] = tot.y;
        offs[4 * n + 2] = tot.z;
        offs[4 * n + 3] = tot.w;
    }
}

// ---- stable counting sort of items by length, longest first (Sec. V.F) ----
constexpr int kSortBlock = 1024;

// The exclusion masks again, in the order the pair kernels read them: word
// (g, lane) holds, for lane (ti, tj) = (lane & 7, lane >> 3), the bits of the
// lane's two pairs (i-atom ti with j-atoms tj and tj + 4) for each i-cluster k
// of group g, at bits 2k and 2k + 1.  A warp then reads one 64-byte row per
// entry instead of one 64-bit mask per i-cluster.
__global__ void k_mask_lanes(long long n_words, const unsigned long long *__restrict__ masks,
                             unsigned short *__restrict__ lanes) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_words) return;
    const long long g = t >> 5;
    const int lane = (int)(t & 31), ti = lane & 7, tj = lane >> 3;
    unsigned w = 0;
#pragma unroll
    for (int k = 0; k < NB_SCL; k++) {
        const unsigned long long m = masks[g * NB_SCL + k];
        w |= (unsigned)((m >> (ti * 8 + tj)) & 1ull) << (2 * k);
        w |= (unsigned)((m >> (ti * 8 + tj + 4)) & 1ull) << (2 * k + 1);
    }
    lanes[t] = (unsigned short)w;
}

__global__ void k_item_hist(int n, int split, const int4 *__restrict__ items, int *__restrict__ hist,
                            int nblk) {
    __shared__ int h[129];
    for (int q = threadIdx.x; q < split; q += blockDim.x) h[q] = 0;
    __syncthreads();
    int i = blockIdx.x * kSortBlock + threadIdx.x;
    if (i < n) atomicAdd(&h[split - items[i].w], 1);
    __syncthreads();
    for (int q = threadIdx.x; q < split; q += blockDim.x) hist[q * nblk + blockIdx.x] = h[q];
}

__global__ void k_scan1(int n, int *__restrict__ v) {  // in-place exclusive scan, one block
    __shared__ int s[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        int i = base + threadIdx.x;
        int x = i < n ? v[i] : 0;
        s[threadIdx.x] = x;
        __syncthreads();
        for (int d = 1; d < blockDim.x; d <<= 1) {
            int t = threadIdx.x >= d ? s[threadIdx.x - d] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < n) v[i] = carry + s[threadIdx.x] - x;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += s[threadIdx.x];
        __syncthreads();
    }
}

__global__ void k_item_scatter(int n, int split, const int4 *__restrict__ in, const int *__restrict__ hist,
                               int nblk, int4 *__restrict__ out) {
    __shared__ int wcount[32][129];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < 32 * 129; t += blockDim.x) (&wcount[0][0])[t] = 0;
    __syncthreads();
    int i = blockIdx.x * kSortBlock + threadIdx.x;
    int q = i < n ? split - in[i].w : 128;
    unsigned peers = __match_any_sync(0xffffffffu, q);
    int rank_w = __popc(peers & ((1u << lane) - 1));
    if (i < n && rank_w == 0) wcount[w][q] = __popc(peers);
    __syncthreads();
    // exclusive scan over warps for each bucket
    for (int b = threadIdx.x; b < split; b += blockDim.x) {
        int acc = 0;
        for (int ww = 0; ww < 32; ww++) {
            int c = wcount[ww][b];
            wcount[ww][b] = acc;
            acc += c;
        }
    }
    __syncthreads();
    if (i < n) out[hist[q * nblk + blockIdx.x] + wcount[w][q] + rank_w] = in[i];
}

}  // namespace

// search units (super-cluster, column segment): the length of the count and offset arrays / 4
int nb_search_segments(const nb_ctx *c) {
    if (c->search_seg > 0) return std::min(c->search_seg, kSegMax);
    int seg = 1;
    while (seg < kSegMax && (long long)c->S_host * seg < kSegWarps) seg *= 2;
    return seg;
}

int nb_search_units(const nb_ctx *c) { return c->S_host * nb_search_segments(c); }

static SearchArgs make_args(nb_ctx *c, float rlist) {
    SearchArgs a;
    a.S = c->S_host;
    a.bb = c->bb;
    a.sbb = c->sbb;
    a.col_sc_off = c->col_sc_off;
    a.ncx = c->ncx;
    a.ncy = c->ncy;
    a.cwx = (float)c->cw[0];
    a.cwy = (float)c->cw[1];
    for (int k = 0; k < 3; k++) a.L[k] = (float)c->box[k];
    // slightly inflated so that FP32 rounding of boxes and shifts cannot drop a pair
    float rs = rlist * (1.0f + 1e-5f) + 1e-5f;
    a.rlist = rs;
    a.rlist2 = rs * rs;
    a.perm = c->perm;
    a.inv = c->inv;
    a.excl_off = c->excl_off;
    a.excl_idx = c->excl_idx;
    a.split = c->split;
    a.seg = nb_search_segments(c);
    a.si_counts = c->si_counts;
    a.si_offs = c->si_offs;
    a.items = c->items_tmp;
    a.cj_out = c->cj_outer;
    a.masks = c->masks;
    return a;
}

nb_status nb_launch_search_count(nb_ctx *c, float rlist, cudaStream_t st) {
    SearchArgs a = make_args(c, rlist);
    const int units = nb_search_units(c);
    int nblk = (units + kWarps - 1) / kWarps;
    c->n_launches += 2;
    k_search<false><<<nblk, kWarps * 32, 0, st>>>(a);
    k_scan4<<<1, 1024, 0, st>>>(units, c->si_counts, c->si_offs);
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}

nb_status nb_launch_search_write(nb_ctx *c, float rlist, cudaStream_t st) {
    SearchArgs a = make_args(c, rlist);
    int nblk = (nb_search_units(c) + kWarps - 1) / kWarps;
    c->n_launches++;
    k_search<true><<<nblk, kWarps * 32, 0, st>>>(a);
    NB_CUDA_TRY(cudaGetLastError());
    if (c->n_masks > 0) {
        const long long words = (long long)c->n_masks * 32;
        c->n_launches++;
        k_mask_lanes<<<(unsigned)((words + 255) / 256), 256, 0, st>>>(words, c->masks, c->mask_lanes);
        NB_CUDA_TRY(cudaGetLastError());
    }
    // order items longest first (stable)
    int n = c->n_items;
    if (n > 0) {
        int nb = (n + kSortBlock - 1) / kSortBlock;
        int *hist = c->sort_tmp;
        c->n_launches += 3;
        k_item_hist<<<nb, kSortBlock, 0, st>>>(n, c->split, c->items_tmp, hist, nb);
        k_scan1<<<1, 1024, 0, st>>>(c->split * nb, hist);
        k_item_scatter<<<nb, kSortBlock, 0, st>>>(n, c->split, c->items_tmp, hist, nb, c->items);
        NB_CUDA_TRY(cudaGetLastError());
    }
    return NB_OK;
}
