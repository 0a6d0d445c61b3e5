// Atom-distance pruning of the cluster pair list (paper Sec. V.D) and the
// dual-list rolling prune (Sec. V.E), plus list diagnostics.
//
// The outer list (bounding-box search at rlist) is kept; the inner list holds,
// for each work item, the outer entries whose interaction-mask bits survive an
// atom-pair distance test at r_in.  A bit k survives iff some atom pair of
// i-cluster k and the j-cluster is closer than r_in at the current positions.
// Rolling: one call prunes the items with index = part (mod n_parts), so the
// whole outer list is re-pruned once every n_parts calls.
#include "nb_pair.cuh"

using namespace nbk;

namespace {

constexpr int kPW = 4;  // warps per block

struct PruneArgs {
    int n_items, part, n_parts;
    const int4 *items;
    const int2 *cj_outer;
    const float4 *xq;
    float Lhi[3], Llo[3];
    float rin2;
    int2 *cj_inner;
    int *inner_len;
    unsigned short *kept;  // [n_j] surviving half masks (lo | hi << 8) per outer entry (scratch)
};

// The rolling prune runs as two kernels so that its parallelism does not depend
// on the length of the work items:
//  k_prune_masks: one warp per chunk of 16 outer entries of an item of this part;
//    the warp works on 4 entries at a time (8 lanes each, lane t of a group owning
//    i-atom t of every i-cluster) and writes each entry's surviving mask byte;
//  k_prune_compact: one warp per item of this part copies the entries whose mask
//    survived, in their original order, into the inner list.
// Items of at most 128 entries (every split nb_set_split allows) are one chunk: the
// warp that prunes an item also compacts it (COMPACT), one launch and no round trip
// of the masks through memory.
constexpr int kPruneChunk = 16;     // entries per warp for items longer than kPruneWhole
constexpr int kPruneWhole = 128;    // items up to this many entries (every split): one warp prunes and compacts them

template <bool COMPACT>
__global__ void __launch_bounds__(kPW * 32) k_prune_masks(PruneArgs a, int chunks_per_item, int chunk) {
    __shared__ float4 s_xi[kPW][NB_SCA];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned full = 0xffffffffu;
    const long long w = (long long)blockIdx.x * kPW + wib;
    const long long item = a.part + (w / chunks_per_item) * a.n_parts;
    if (item >= a.n_items) return;
    const int4 it = a.items[item];
    const int e_begin = (int)(w % chunks_per_item) * chunk;
    if (e_begin >= it.w) {
        if (COMPACT && lane == 0) a.inner_len[item] = 0;
        return;
    }
    const int e_end = min(it.w, e_begin + chunk);
    const int si = it.x, sidx = it.y, j0 = it.z;
    const ShiftSplit sh = make_shift(sidx, a.Lhi, a.Llo);
    for (int h = 0; h < 2; h++) {
        int at = lane + 32 * h;
        s_xi[wib][at] = shift_i(a.xq[si * NB_SCA + at], sh);
    }
    __syncwarp();
    const int g = lane >> 3, t = lane & 7;
    int cnt = 0;  // COMPACT: entries kept so far
    for (int e0 = e_begin; e0 < e_end; e0 += 4) {
        const int e = e0 + g;
        const bool valid = e < e_end;
        const int2 ent = valid ? a.cj_outer[j0 + e] : make_int2(0, 0);
        const int im = ent.y & 0xff;
        // j-atoms b and b + 4 as packed pairs: component 0 decides the lower j-half,
        // component 1 the upper
        float2 jx[4], jy[4], jz[4];
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const float4 p0 = shift_j(a.xq[ent.x * NB_CL + b], sh), p1 = shift_j(a.xq[ent.x * NB_CL + b + 4], sh);
            jx[b] = make_float2(p0.x, p1.x);
            jy[b] = make_float2(p0.y, p1.y);
            jz[b] = make_float2(p0.z, p1.z);
        }
        int lo = 0, hi = 0;
#pragma unroll
        for (int k = 0; k < NB_SCL; k++) {
            if (im & (1 << k)) {
                const float4 xi = s_xi[wib][k * NB_CL + t];
                // q = r^2 - r_in^2 in one FMA chain: a pair is inside iff q's sign bit is set,
                // so the test of 8 pairs is a bitwise OR (r_in carries a margin of 2e-6, far
                // above the rounding of q, so every pair closer than r_in is kept)
                unsigned s0 = 0u, s1 = 0u;
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    const float2 dx = psub(p2(xi.x), jx[b]), dy = psub(p2(xi.y), jy[b]), dz = psub(p2(xi.z), jz[b]);
                    const float2 q = pfma(dz, dz, pfma(dy, dy, pfma(dx, dx, p2(-a.rin2))));
                    s0 |= __float_as_uint(q.x);
                    s1 |= __float_as_uint(q.y);
                }
                lo |= (int)(s0 >> 31) << k;
                hi |= (int)(s1 >> 31) << k;
            }
        }
        int kept = lo | (hi << 8);
        kept |= __shfl_xor_sync(full, kept, 1);
        kept |= __shfl_xor_sync(full, kept, 2);
        kept |= __shfl_xor_sync(full, kept, 4);
        if (COMPACT) {
            // lane 0 of each group holds its entry's masks; entries keep their order
            const bool keep = t == 0 && valid && kept != 0;
            const unsigned kb = __ballot_sync(full, keep);
            if (keep)
                a.cj_inner[j0 + cnt + __popc(kb & ((1u << lane) - 1))] =
                    make_int2(ent.x | ((kept >> 8) << 24), (ent.y & ~0xff) | (kept & 0xff));
            cnt += __popc(kb);
        } else if (t == 0 && valid) {
            a.kept[j0 + e] = (unsigned short)kept;
        }
    }
    if (COMPACT && lane == 0) a.inner_len[item] = cnt;
}

__global__ void __launch_bounds__(kPW * 32) k_prune_compact(PruneArgs a) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned full = 0xffffffffu;
    const long long w = (long long)blockIdx.x * kPW + wib;
    const long long item = a.part + w * a.n_parts;
    if (item >= a.n_items) return;
    const int4 it = a.items[item];
    const int j0 = it.z, len = it.w;
    int cnt = 0;
    for (int e0 = 0; e0 < len; e0 += 32) {
        const int e = e0 + lane;
        int kept = 0;
        int2 ent = make_int2(0, 0);
        if (e < len) {
            kept = a.kept[j0 + e];
            if (kept) ent = a.cj_outer[j0 + e];
        }
        const unsigned keep = __ballot_sync(full, kept != 0);
        if (kept)
            a.cj_inner[j0 + cnt + __popc(keep & ((1u << lane) - 1))] =
                make_int2(ent.x | ((kept >> 8) << 24), (ent.y & ~0xff) | (kept & 0xff));
        cnt += __popc(keep);
    }
    if (lane == 0) a.inner_len[item] = cnt;
}

// Counts over a list (inner_len == nullptr: the outer list): pairs inside rc that are
// computed, and 64 per mask bit.
__global__ void __launch_bounds__(kPW * 32)
    k_count(int n_items, const int4 *items, const int *inner_len, const int2 *cj, const unsigned long long *masks,
            const float4 *xq, float Lhi0, float Lhi1, float Lhi2, float Llo0, float Llo1, float Llo2, float rc2,
            unsigned long long *out) {
    __shared__ float4 s_xi[kPW][NB_SCA];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int item = blockIdx.x * kPW + wib;
    if (item >= n_items) return;
    const float Lhi[3] = {Lhi0, Lhi1, Lhi2}, Llo[3] = {Llo0, Llo1, Llo2};
    const int4 it = items[item];
    const int len = inner_len ? inner_len[item] : it.w;
    const ShiftSplit sh = make_shift(it.y, Lhi, Llo);
    for (int h = 0; h < 2; h++) {
        int at = lane + 32 * h;
        s_xi[wib][at] = shift_i(xq[it.x * NB_SCA + at], sh);
    }
    __syncwarp();
    const int ti = lane & 7, tj = lane >> 3;
    unsigned long long within = 0, evald = 0;
    const bool is_inner = inner_len != nullptr;
    for (int e = 0; e < len; e++) {
        const int2 ent = cj[it.z + e];
        // outer entries: one mask bit per i-cluster for the whole j-cluster;
        // inner entries: one bit per (i-cluster, j-half)
        const int c = is_inner ? inner_cj(ent) : ent.x, mg = entry_group(ent);
        const int lo = ent.y & 0xff, hi = is_inner ? inner_hi(ent) : lo;
        for (int k = 0; k < NB_SCL; k++) {
            if (!((lo | hi) >> k & 1)) continue;
            const unsigned long long m = mg ? masks[(size_t)(mg - 1) * 8 + k] : ~0ull;
            const float4 xi = s_xi[wib][k * NB_CL + ti];
            for (int h = 0; h < 2; h++) {
                if (!(((h ? hi : lo) >> k) & 1)) continue;
                evald += 1;
                const float4 xj = shift_j(xq[c * NB_CL + tj + 4 * h], sh);
                float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
                float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                bool bit = (m >> (ti * 8 + tj + 4 * h)) & 1ull;
                within += (bit && r2 < rc2) ? 1 : 0;
            }
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        within += __shfl_xor_sync(0xffffffffu, within, d);
        evald += __shfl_xor_sync(0xffffffffu, evald, d);
    }
    if (lane == 0) {
        atomicAdd(&out[0], within);
        atomicAdd(&out[1], evald);
    }
}

// Export of atom pairs (caller indices and image shifts) for set mask bits.
__global__ void __launch_bounds__(kPW * 32)
    k_export(int n_items, const int4 *items, const int *inner_len, const int2 *cj,
             const unsigned long long *masks, const int *perm, const int *img, long long cap,
             long long *buf, unsigned long long *count) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int item = blockIdx.x * kPW + wib;
    if (item >= n_items) return;
    const int4 it = items[item];
    const int len = inner_len ? inner_len[item] : it.w;
    int sx, sy, sz;
    shift_of(it.y, sx, sy, sz);
    for (int e = 0; e < len; e++) {
        const int2 ent = cj[it.z + e];
        const bool is_inner = inner_len != nullptr;
        const int c = is_inner ? inner_cj(ent) : ent.x, mg = entry_group(ent);
        const int lo = ent.y & 0xff, hi = is_inner ? inner_hi(ent) : lo;
        for (int k = 0; k < NB_SCL; k++) {
            if (!((lo | hi) >> k & 1)) continue;
            const unsigned long long m = mg ? masks[(size_t)(mg - 1) * 8 + k] : ~0ull;
            for (int h = 0; h < 2; h++) {
                const int p = lane + 32 * h;  // p = 8*a + b
                const int ia = p >> 3, jb = p & 7;
                if (!((m >> p) & 1ull)) continue;
                if (!((((jb < 4) ? lo : hi) >> k) & 1)) continue;
                const int i = perm[it.x * NB_SCA + k * NB_CL + ia];
                const int j = perm[c * NB_CL + jb];
                if (i < 0 || j < 0) continue;
                int ix, iy, iz, jx, jy, jz;
                img_unpack(img[i], ix, iy, iz);
                img_unpack(img[j], jx, jy, jz);
                unsigned long long slot = atomicAdd(count, 1ull);
                if ((long long)slot < cap) {
                    long long *o = buf + 5 * slot;
                    o[0] = i;
                    o[1] = j;
                    o[2] = sx - ix + jx;
                    o[3] = sy - iy + jy;
                    o[4] = sz - iz + jz;
                }
            }
        }
    }
}

void box_split(const nb_ctx *c, float *hi, float *lo) {
    for (int k = 0; k < 3; k++) {
        hi[k] = (float)c->box[k];
        lo[k] = (float)(c->box[k] - (double)hi[k]);
    }
}

}  // namespace

nb_status nb_launch_prune(nb_ctx *c, float r_in, int part, int n_parts, cudaStream_t st) {
    if (c->n_items == 0) return NB_OK;
    PruneArgs a;
    a.n_items = c->n_items;
    a.part = part;
    a.n_parts = n_parts;
    a.items = c->items;
    a.cj_outer = c->cj_outer;
    a.xq = nb_cur_xq(c);
    box_split(c, a.Lhi, a.Llo);
    // a hair wider than r_in so that FP32 rounding never drops a pair the FP64 definition keeps
    float re = r_in * (1.0f + 2e-6f);
    a.rin2 = re * re;
    a.cj_inner = c->cj_inner;
    a.inner_len = c->inner_len;
    a.kept = c->kept;
    long long nw = (c->n_items - part + n_parts - 1) / n_parts;
    if (nw <= 0) return NB_OK;
    // items of at most kPruneWhole entries: one warp per item, pruned and compacted in one
    // pass; longer ones: chunks of kPruneChunk entries, then a compaction kernel
    const int chunk = c->split_built <= kPruneWhole ? std::max(c->split_built, 1) : kPruneChunk;
    const int chunks = (c->split_built + chunk - 1) / chunk;
    NbTraceScope tr(c, NB_TRACE_PRUNE, st);
    c->n_launches += 2;
    const long long nwm = nw * chunks;
    if (chunks == 1) {  // an item fits one chunk: prune and compact in one pass
        c->n_launches--;
        k_prune_masks<true><<<(unsigned)((nwm + kPW - 1) / kPW), kPW * 32, 0, st>>>(a, chunks, chunk);
    } else {
        k_prune_masks<false><<<(unsigned)((nwm + kPW - 1) / kPW), kPW * 32, 0, st>>>(a, chunks, chunk);
        k_prune_compact<<<(unsigned)((nw + kPW - 1) / kPW), kPW * 32, 0, st>>>(a);
    }
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}

// Compaction of every item's outer entries by the masks in c->kept (after the
// fused first-use prune of the force kernel).
nb_status nb_launch_prune_compact_all(nb_ctx *c, cudaStream_t st) {
    if (c->n_items == 0) return NB_OK;
    PruneArgs a;
    a.n_items = c->n_items;
    a.part = 0;
    a.n_parts = 1;
    a.items = c->items;
    a.cj_outer = c->cj_outer;
    a.xq = c->xq;
    box_split(c, a.Lhi, a.Llo);
    a.rin2 = 0.f;
    a.cj_inner = c->cj_inner;
    a.inner_len = c->inner_len;
    a.kept = c->kept;
    c->n_launches++;
    k_prune_compact<<<(unsigned)((c->n_items + kPW - 1) / kPW), kPW * 32, 0, st>>>(a);
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}

// Calls that need the inner list while its fused first-use prune is still
// pending prune the whole outer list first, at the positions of the last sort
// or force call.
nb_status nb_ensure_inner(nb_ctx *c, cudaStream_t st) {
    if (!c->inner_pending) return NB_OK;
    const nb_status s = nb_launch_prune(c, (float)c->r_in, 0, 1, st);
    if (s == NB_OK) c->inner_pending = false;
    return s;
}

nb_status nb_launch_count(nb_ctx *c, int which, cudaStream_t st) {
    NB_CUDA_TRY(cudaMemsetAsync(c->diag, 0, 2 * sizeof(long long), st));
    if (c->n_items == 0) return NB_OK;
    float hi[3], lo[3];
    box_split(c, hi, lo);
    float rc = (float)c->rc;
    c->n_launches++;
    k_count<<<(c->n_items + kPW - 1) / kPW, kPW * 32, 0, st>>>(
        c->n_items, c->items, which == NB_LIST_INNER ? c->inner_len : nullptr,
        which == NB_LIST_INNER ? c->cj_inner : c->cj_outer, c->masks, nb_cur_xq(c), hi[0], hi[1], hi[2], lo[0], lo[1],
        lo[2], rc * rc, reinterpret_cast<unsigned long long *>(c->diag));
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}

nb_status nb_launch_export(nb_ctx *c, int which, long long *buf, long long cap, long long *count,
                           cudaStream_t st) {
    NB_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(long long), st));
    if (c->n_items == 0) return NB_OK;
    const bool inner = which == NB_LIST_INNER;
    c->n_launches++;
    k_export<<<(c->n_items + kPW - 1) / kPW, kPW * 32, 0, st>>>(
        c->n_items, c->items, inner ? c->inner_len : nullptr, inner ? c->cj_inner : c->cj_outer, c->masks,
        c->perm, c->img, cap, buf, reinterpret_cast<unsigned long long *>(count));
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}
