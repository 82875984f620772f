// walk.cu -- interaction lists: one warp walks the tree for one i-group.
//
// The Barnes-Hut traversal with a fixed opening angle (Sect. 3.2), done
// once per i-group as in the modified tree algorithm of Barnes (1990) that
// the paper's cost model uses (Sect. 5.5, T_icalc,const).  The paper does
// not state the criterion; this library opens a cell C for group G iff
//   (a) C's grid cube meets G's grid box (closed integer intervals of the
//       quantised coordinates), or
//   (b) ell_C^2 >= theta^2 d^2, ell_C = L 2^-level, d = distance from C's
//       centre of mass to G's FP64 bounding box,
// and evaluates (b) as FP64 with each operation rounded on its own, in a
// fixed order.  The same FP64 decision is reproduced here at FP32 cost: the
// test is first evaluated in FP32 on double-float (hi + lo) copies of the
// positions relative to the group centre, with a rigorous bound on the
// FP32 error; only tests that land inside that bound are re-evaluated with
// the exact FP64 operation sequence.
//
// Traversal is breadth-first per warp: 32 cells of the current frontier are
// tested at a time; opened internal cells push their children (contiguous
// ids) to the next frontier, opened leaves append one EPJ entry (node id
// with bit 31 set: all of the leaf's particles), unopened cells one SPJ
// entry.  A group's list is contiguous in a pool handed out in chunks of at
// least 2^16 entries; when a chunk fills, the group's partial list moves to
// a fresh chunk twice its length.  Overflow of the pool or of the frontier sets a flag; the
// host then grows the buffer and repeats the walk.
#include "fdps_internal.cuh"

namespace fdps {

struct WalkArgs {
    DevState* st;
    const uint32_t* nd_count;
    const uint4* nd_walk;  // (q_x | level, leaf, children; q_y; q_z; first child | leaf count)
    const float4* nd_f;    // COM hi/lo pairs per node
    const dvec4* nd_com;
    const uint32_t* g_count;
    const uint32_t* g_first;
    const uint32_t* sys;  // system of each particle position (null: one system)
    const SysBox* box;    // root box of each system
    const uint32_t* g_qbox;
    const double* g_box;
    const float4* g_ch;
    const float4* g_cl;
    const float4* g_blo;
    const float4* g_bhi;
    unsigned long long* g_off;
    uint32_t* g_len;
    uint32_t* g_nspj;
    uint32_t* g_nepj;
    uint32_t* pool;
    unsigned long long cap_pool;
    uint32_t* frontier;
    uint32_t cap_frontier;
    double theta2;
    float theta2f;
};

namespace {

constexpr unsigned long long kChunk = 1ull << 16;
constexpr float kU32 = 5.9604645e-08f;  // 2^-24, unit roundoff of FP32

__device__ __forceinline__ unsigned long long shfl_u64(unsigned long long v, int src) {
    return __shfl_sync(0xFFFFFFFFu, v, src);
}

// Exact FP64 opening test (b): the reference sequence of operations.
__device__ __forceinline__ bool open_fp64(double L, int level, double theta2, const dvec4 com,
                                       const double* box) {
    const double ell = ldexp(L, -level);
    const double c[3] = {com.x, com.y, com.z};
    double d2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double below = __dsub_rn(box[a], c[a]);
        const double above = __dsub_rn(c[a], box[3 + a]);
        const double da = below > 0.0 ? below : (above > 0.0 ? above : 0.0);
        d2 = __dadd_rn(d2, __dmul_rn(da, da));
    }
    return __dmul_rn(ell, ell) >= __dmul_rn(theta2, d2);
}

// What a warp carries from one group's walk to the next: its pool chunk
// and its totals for the device state word.  Every field is the same in
// all lanes.
struct WalkState {
    unsigned long long cbase;  // start of the warp's pool chunk
    uint32_t coff, clen;       // cursor and length within it
    bool ovf;
    unsigned long long acc_entries, acc_epj, acc_spj, acc_iepj, acc_ispj;
    uint32_t max_front;
};

__device__ __forceinline__ WalkState walk_state_init() {
    WalkState S;
    S.cbase = 0;
    S.coff = S.clen = 0;
    S.ovf = false;
    S.acc_entries = S.acc_epj = S.acc_spj = S.acc_iepj = S.acc_ispj = 0;
    S.max_front = 0;
    return S;
}


// The list of group g, walked by the calling warp (all 32 lanes), with its
// two frontier buffers fa and fb and the warp's per-level thresholds thr.
__device__ __forceinline__ void walk_group(const WalkArgs& A, uint32_t g, uint32_t* fa, uint32_t* fb,
                                           float2* thr, WalkState& S) {
    DevState* st = A.st;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t F = A.cap_frontier;
    // the group's system: its root node (node id = system index) and box
    const uint32_t sysid = A.sys ? A.sys[A.g_first[g]] : 0u;
    const double L = A.box[sysid].L;
    const float Lf = __double2float_rn(L);
    // the FP32 filter's bound holds while the squares of cell sizes stay
    // normal FP32 numbers (with or without flushing of subnormals): outside
    // this range of root boxes every test takes the exact FP64 sequence
    const bool filt = Lf >= 0x1p-40f && Lf <= 0x1p60f;
    const uint32_t* qb = A.g_qbox + 6 * (int64_t)g;
    const uint32_t qmin0 = qb[0], qmin1 = qb[1], qmin2 = qb[2];
    const uint32_t qmax0 = qb[3], qmax1 = qb[4], qmax2 = qb[5];
    const float4 gch = A.g_ch[g], gcl = A.g_cl[g];
    const float4 blo = A.g_blo[g], bhi = A.g_bhi[g];
    const float hb = fmaxf(fmaxf(fmaxf(-blo.x, -blo.y), fmaxf(-blo.z, bhi.x)), fmaxf(bhi.y, bhi.z));
    const double* box64 = A.g_box + 6 * (int64_t)g;
    // Coefficients of the filter's error bound as a polynomial in M = max|d| +
    // hb (d the FP32 offset of a cell's centre of mass, hb the largest
    // |corner| of the group box): with E = 4uM + e0 the error of one
    // coordinate and S1 = t_x + t_y + t_z <= 3M, theta^2 (2 E S1 + 3 E^2) <=
    // theta^2 (25 u M^2 + 7 e0 M + 4 e0^2); 1 % on top covers the rounding of
    // the bound's own FP32 evaluation.
    const float e0 = 1e-13f * Lf;
    const float mc1 = 1.01f * A.theta2f * 25.0f * kU32, mc2 = 1.01f * A.theta2f * 7.0f * e0,
                mc3 = 1.01f * A.theta2f * 4.0f * e0 * e0;
    // The bound's largest value over the cells each side can decide, as two
    // thresholds on d^2 per level (lane = level): a cell with d^2 <= D0^2 =
    // ell^2 / theta^2 has M <= D0 + 2 hb (|d_a| <= t_a + hb), so the margin
    // is at most Mo and d^2 < (ell^2 - Mo) / theta^2 opens it; beyond D0,
    // with (s + 2 hb)^2 <= 2 s^2 + 8 hb^2 and s = |t| <= (d^2 + D0^2) / (2 D0),
    // the margin is linear in d^2 and d^2 above hi rejects it.  Slack covers
    // the thresholds' own FP32 evaluation; outside the filter's range of L
    // (and at theta = 0, where every cell opens) no threshold decides.
    __syncwarp();  // the previous group's walk has read thr
    if (lane <= kMaxLevel) {
        float lo = -INFINITY, hi = INFINITY;
        if (!filt) {
        } else if (A.theta2f == 0.0f) {
            lo = INFINITY;
        } else {
            const float ell = __int_as_float(__float_as_int(Lf) - (lane << 23));
            const float l2 = ell * ell;
            const float D0 = sqrtf(l2 / A.theta2f);
            const float Mb = D0 + 2.0f * hb;
            const float Mo = fmaf(16.0f * kU32, l2, fmaf(fmaf(mc1, Mb, mc2), Mb, mc3));
            lo = (l2 - Mo) / A.theta2f * (1.0f - 8.0f * kU32);
            const float coef = A.theta2f - (8.0f * kU32 * A.theta2f + 2.0f * mc1 + mc2 / (2.0f * D0));
            const float rhs = l2 * (1.0f + 8.0f * kU32) + 8.0f * mc1 * hb * hb + mc2 * (0.5f * D0 + 2.0f * hb) + mc3;
            if (coef > 0.0f) hi = rhs * (1.0f + 16.0f * kU32) / coef;
        }
        thr[lane] = make_float2(lo, hi);
    }
    __syncwarp();

    if (S.ovf) {  // counting only: keep the in-chunk cursor small
        S.cbase += S.coff;
        S.coff = 0;
    }
    unsigned long long gstart = S.cbase + S.coff;
    uint32_t* cptr = A.pool + S.cbase;
    uint32_t nspj = 0, nepj_lane = 0;
    uint32_t fsize = 1;
    if (lane == 0) fa[0] = sysid;
    __syncwarp();
    while (fsize > 0) {
        uint32_t nsize = 0;
        S.max_front = fsize > S.max_front ? fsize : S.max_front;
        // the first batch's frontier entries, node records and COM pairs;
        // every batch then fetches the next one's before testing its own
        // (frontier ids two batches ahead, records one batch ahead, so
        // no batch waits on a load that depends on another load)
        uint32_t node_nx = lane < fsize ? fa[lane] : 0u;
        uint32_t node_nx2 = lane + 32 < fsize ? fa[lane + 32] : 0u;
        uint4 rec_nx = make_uint4(0, 0, 0, 0);
        float4 fh_nx = make_float4(0.f, 0.f, 0.f, 0.f), fl_nx = fh_nx;
        if (lane < fsize) {
            rec_nx = A.nd_walk[node_nx];
            fh_nx = A.nd_f[2 * node_nx];
            fl_nx = A.nd_f[2 * node_nx + 1];
        }
        for (uint32_t base = 0; base < fsize; base += 32) {
            const uint32_t idx = base + lane;
            const bool act = idx < fsize;
            const uint32_t node = node_nx;
            const uint4 rec = rec_nx;
            const float4 fh = fh_nx, fl = fl_nx;
            if (idx + 32 < fsize) {
                node_nx = node_nx2;
                rec_nx = A.nd_walk[node_nx];
                fh_nx = A.nd_f[2 * node_nx];
                fl_nx = A.nd_f[2 * node_nx + 1];
            }
            if (idx + 64 < fsize) node_nx2 = fa[idx + 64];
            int action = 0;  // 1 SPJ, 2 EPJ leaf, 3 open internal
            uint32_t nch = 0, child = 0;
            if (act) {
                const int level = (int)((rec.x >> 21) & 31u);
                const bool leaf = (rec.x >> 26) & 1u;
                const uint32_t w = (1u << (kMaxLevel - level)) - 1u;
                const uint32_t qx = rec.x & kQMax, qy = rec.y, qz = rec.z;
                const bool meets = qx <= qmax0 && qx + w >= qmin0 && qy <= qmax1 &&
                                   qy + w >= qmin1 && qz <= qmax2 && qz + w >= qmin2;
                bool open = true;
                if (!meets) {
                    const float dx = (fh.x - gch.x) + (fl.x - gcl.x);
                    const float dy = (fh.y - gch.y) + (fl.y - gcl.y);
                    const float dz = (fh.z - gch.z) + (fl.z - gcl.z);
                    const float tx = fmaxf(fmaxf(blo.x - dx, dx - bhi.x), 0.0f);
                    const float ty = fmaxf(fmaxf(blo.y - dy, dy - bhi.y), 0.0f);
                    const float tz = fmaxf(fmaxf(blo.z - dz, dz - bhi.z), 0.0f);
                    const float d2 = tx * tx + ty * ty + tz * tz;
                    const float2 th = thr[level];
                    if (d2 < th.x) {
                        open = true;
                    } else if (d2 > th.y) {
                        open = false;
                    } else {
                        open = open_fp64(L, level, A.theta2, A.nd_com[node], box64);
                        atomicAdd(&st->fallbacks, 1ull);  // rare: counted where it happens
                    }
                }
                if (!open) {
                    action = 1;
                } else if (leaf) {
                    action = 2;
                    nepj_lane += rec.w;  // the leaf's particle count
                } else {
                    action = 3;
                    child = rec.w;
                    nch = rec.x >> 27;
                }
            }
            // ---- append SPJ / EPJ entries
            const bool emit = action == 1 || action == 2;
            const uint32_t emask = __ballot_sync(0xFFFFFFFFu, emit);
            const uint32_t k = __popc(emask);
            if (k) {
                if (S.coff + k > S.clen) {
                    // new chunk: at least kChunk entries and twice the
                    // group's list so far, so long lists move O(log) times
                    const unsigned long long sofar = S.cbase + S.coff - gstart;
                    const unsigned long long want =
                        2 * (sofar + k) > kChunk ? 2 * (sofar + k) : kChunk;
                    unsigned long long nb = 0;
                    if (lane == 0) nb = atomicAdd(&st->pool_cursor, want);
                    nb = shfl_u64(nb, 0);
                    if (!S.ovf && (nb + want > A.cap_pool || want > 0xFFFFFFFFull)) {
                        if (lane == 0) atomicOr(&st->overflow, kOvfPool);
                        S.ovf = true;
                    }
                    if (!S.ovf) {
                        for (unsigned long long j = lane; j < sofar; j += 32)
                            A.pool[nb + j] = A.pool[gstart + j];
                        __syncwarp();
                        gstart = nb;
                        S.cbase = nb;
                        S.coff = (uint32_t)sofar;
                        S.clen = (uint32_t)want;
                        cptr = A.pool + nb;
                    } else {
                        // count only from here on
                        S.cbase = gstart;
                        S.coff = (uint32_t)sofar;
                        S.clen = 0xFFFFFFFFu;
                    }
                }
                if (emit && !S.ovf) cptr[S.coff + __popc(emask & lt)] = action == 2 ? (node | kLeafTag) : node;
                S.coff += k;
            }
            nspj += __popc(__ballot_sync(0xFFFFFFFFu, action == 1));
            // ---- push children of opened internal cells (deep in the
            // tree most batches open none)
            if (__ballot_sync(0xFFFFFFFFu, nch > 0u)) {
                uint32_t inc = nch;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    uint32_t tv = __shfl_up_sync(0xFFFFFFFFu, inc, off);
                    if (lane >= off) inc += tv;
                }
                const uint32_t tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
                if (nsize + tot > F) {
                    if (lane == 0) atomicOr(&st->overflow, kOvfFrontier);
                    S.ovf = true;
                } else {
                    const uint32_t o = nsize + inc - nch;
                    for (uint32_t c = 0; c < nch; ++c) fb[o + c] = child + c;
                    nsize += tot;
                }
            }
        }
        __syncwarp();
        uint32_t* tmp = fa;
        fa = fb;
        fb = tmp;
        fsize = nsize;
    }
    const uint32_t nepj = __reduce_add_sync(0xFFFFFFFFu, nepj_lane);
    const unsigned long long len = S.cbase + S.coff - gstart;
    if (lane == 0) {
        A.g_off[g] = gstart;
        A.g_len[g] = (uint32_t)len;
        A.g_nspj[g] = nspj;
        A.g_nepj[g] = nepj;
    }
    const unsigned long long ni = A.g_count[g];
    S.acc_entries += len;
    S.acc_epj += nepj;
    S.acc_spj += nspj;
    S.acc_iepj += ni * nepj;
    S.acc_ispj += ni * nspj;
}

// The warp's totals into the device state word (lane 0).
__device__ __forceinline__ void walk_flush(const WalkArgs& A, const WalkState& S) {
    DevState* st = A.st;
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&st->pool_needed, S.acc_entries);
        atomicAdd(&st->list_entries, S.acc_entries);
        atomicAdd(&st->n_epj, S.acc_epj);
        atomicAdd(&st->n_spj, S.acc_spj);
        atomicAdd(&st->int_epj, S.acc_iepj);
        atomicAdd(&st->int_spj, S.acc_ispj);
        atomicMax(&st->max_frontier, S.max_front);
    }
}

constexpr int kWalkBlock = 128;

__global__ void __launch_bounds__(kWalkBlock, 8) k_walk(WalkArgs A) {
    DevState* st = A.st;
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    uint32_t* fa = A.frontier + wid * 2 * (int64_t)A.cap_frontier;
    uint32_t* fb = fa + A.cap_frontier;
    const uint32_t ngroups = (uint32_t)st->n_groups;
    __shared__ float2 s_thr[kWalkBlock / 32][kMaxLevel + 1];
    WalkState S = walk_state_init();
    for (;;) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(&st->walk_counter, 1u);
        g = __shfl_sync(0xFFFFFFFFu, g, 0);
        if (g >= ngroups) break;
        walk_group(A, g, fa, fb, s_thr[threadIdx.x >> 5], S);
    }
    walk_flush(A, S);
}

}  // namespace

int walk_blocks(fdps_ctx* ctx) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk, kWalkBlock, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 4;
    return per_sm * ctx->sm_count;
}

int walk_warps_per_block() { return kWalkBlock / 32; }

unsigned long long walk_chunk() { return kChunk; }

WalkArgs walk_args(fdps_tree* t, const uint32_t* sys) {
    WalkArgs A;
    A.st = t->st;
    A.nd_count = t->nd_count;
    A.nd_walk = t->nd_walk;
    A.nd_f = t->nd_f;
    A.nd_com = t->nd_com;
    A.g_count = t->g_count;
    A.g_first = t->g_first;
    A.sys = sys;
    A.box = t->sys_box;
    A.g_qbox = t->g_qbox;
    A.g_box = t->g_box;
    A.g_ch = t->g_ch;
    A.g_cl = t->g_cl;
    A.g_blo = t->g_blo;
    A.g_bhi = t->g_bhi;
    A.g_off = t->g_off;
    A.g_len = t->g_len;
    A.g_nspj = t->g_nspj;
    A.g_nepj = t->g_nepj;
    A.pool = t->pool;
    A.cap_pool = (unsigned long long)t->cap_pool;
    A.frontier = t->frontier;
    A.cap_frontier = (uint32_t)t->cap_frontier;
    A.theta2 = t->p.theta * t->p.theta;
    A.theta2f = (float)A.theta2;
    return A;
}

int launch_walk(fdps_tree* t, const uint32_t* sys, int blocks) {
    fdps_ctx* ctx = t->ctx;
    const WalkArgs A = walk_args(t, sys);
    k_walk<<<blocks, kWalkBlock, 0, ctx->stream>>>(A);
    FDPS_LAUNCH_CHECK(ctx);
    return FDPS_OK;
}

}  // namespace fdps
