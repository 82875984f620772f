// short.cu -- the short-range mode: neighbour search over the same tree.
//
// FDPS treats an interaction as short-range when it has a cutoff and finds
// the neighbours by a tree traversal (Sect. 2.1.2, 3.2), for four kinds of
// cutoff: fixed, j-dependent, i-dependent and symmetric.  Particle j is a
// neighbour of i (i itself included) iff r^2 < c^2, with r^2 evaluated in
// FP64 as (dx*dx + dy*dy) + dz*dz, each operation rounded on its own, and
//   fixed: c = r_fixed;  i-dependent: c = h_i;  j-dependent: c = h_j;
//   symmetric: c = max(h_i, h_j).
// The workload on the neighbours is the SPH density with the Wendland C6
// kernel of the paper's SPH runs (Sect. 4.3): rho_i = sum_j m_j W(r, H),
// H = r_fixed, h_i or h_j, and for the symmetric cutoff the mean of
// W(r, h_i) and W(r, h_j).
//
// Per i-group, a warp walks the tree from the system's root and keeps every
// leaf that may hold a neighbour: a cell is opened iff the smallest distance
// between its grid cube and the group's grid box (an exact lower bound in
// grid units) is below the largest cutoff that can apply (r_fixed, the
// group's largest h, the cell's largest h, or both), with a relative margin
// so that no neighbour's leaf is ever dropped.  The pair pass then decides
// each candidate pair exactly: an FP32 evaluation on hi/lo parts with a
// bound on its error settles all but the pairs within the bound of the
// cutoff, which are decided by the FP64 operation sequence above.
#include "fdps_internal.cuh"

namespace fdps {
namespace {

constexpr int kSBlock = 128;
constexpr int kSW = kSBlock / 32;
constexpr int kSTile = 64;                 // candidate particles per shared tile
constexpr unsigned long long kSChunk = 1ull << 16;
constexpr float kU = 5.9604645e-08f;      // 2^-24
// Wendland C6, 3D, support H: W = 1365 / (64 pi H^3) (1-q)^8 (1 + 8q + 25q^2 + 32q^3)
constexpr float kWc6 = 6.7889530f;        // 1365 / (64 pi)

__global__ void k_short_h(int64_t n, const uint32_t* __restrict__ id, const double* __restrict__ h_user,
                          double* __restrict__ h_sorted, uint32_t* flag) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double h = h_user[id[p]];
        if (!(h > 0.0) || !(h < 1e300)) atomicOr(flag, 1u);
        h_sorted[p] = h;
    }
}

__global__ void k_hmax_leaves(int64_t nn, const uint32_t* __restrict__ meta, const uint32_t* __restrict__ first,
                              const uint32_t* __restrict__ count, const double* __restrict__ h,
                              double* __restrict__ hmax) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!((meta[i] >> 16) & 1u)) continue;
        double m = 0.0;
        for (uint32_t p = first[i]; p < first[i] + count[i]; ++p) m = h[p] > m ? h[p] : m;
        hmax[i] = m;
    }
}

__global__ void k_hmax_internal(int64_t a, int64_t b, const uint32_t* __restrict__ meta,
                                const uint32_t* __restrict__ child, double* __restrict__ hmax) {
    for (int64_t i = a + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t mt = meta[i];
        if ((mt >> 16) & 1u) continue;
        const uint32_t c0 = child[i], nc = (mt >> 8) & 0xFFu;
        double m = 0.0;
        for (uint32_t c = c0; c < c0 + nc; ++c) m = hmax[c] > m ? hmax[c] : m;
        hmax[i] = m;
    }
}

__global__ void k_group_hmax(int64_t ng, const uint32_t* __restrict__ first, const uint32_t* __restrict__ count,
                             const double* __restrict__ h, double* __restrict__ ghmax) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng;
         g += (int64_t)gridDim.x * blockDim.x) {
        double m = 0.0;
        for (uint32_t p = first[g]; p < first[g] + count[g]; ++p) m = h[p] > m ? h[p] : m;
        ghmax[g] = m;
    }
}

struct ShortWalkArgs {
    DevState* st;
    const uint4* nd_walk;  // (q_x | level, leaf, children; q_y; q_z; first child | leaf count)
    const double* nd_hmax;
    const uint32_t* g_qbox;
    const uint32_t* g_first;
    const double* g_hmax;
    const uint32_t* sys;
    const SysBox* box;
    unsigned long long* g_off;
    uint32_t* g_len;
    uint32_t* g_nepj;  // candidate particles per group
    uint32_t* pool;
    unsigned long long cap_pool;
    uint32_t* frontier;
    uint32_t cap_frontier;
    int mode;
    float r_fixed;
};

// cutoff bound for a cell (cell's largest h) and a group (group's largest h)
__device__ __forceinline__ float short_bound(int mode, float r_fixed, float hcell, float hgroup) {
    return mode == 0 ? r_fixed : mode == 1 ? hgroup : mode == 2 ? hcell : fmaxf(hcell, hgroup);
}

__global__ void __launch_bounds__(kSBlock) k_short_walk(ShortWalkArgs A) {
    DevState* st = A.st;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    uint32_t* fa = A.frontier + wid * 2 * (int64_t)A.cap_frontier;
    uint32_t* fb = fa + A.cap_frontier;
    const uint32_t F = A.cap_frontier;
    const uint32_t ngroups = (uint32_t)st->n_groups;
    unsigned long long cursor = 0, chunk_end = 0, acc_entries = 0, acc_cand = 0;
    bool ovf = false;
    for (;;) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(&st->walk_counter, 1u);
        g = __shfl_sync(0xFFFFFFFFu, g, 0);
        if (g >= ngroups) break;
        const uint32_t sysid = A.sys ? A.sys[A.g_first[g]] : 0u;
        // grid spacing of the system, squared, in FP32
        const float dq = (float)(A.box[sysid].L * (1.0 / 2097152.0));
        const float dq2 = dq * dq;
        const uint32_t* qb = A.g_qbox + 6 * (int64_t)g;
        const uint32_t qmin0 = qb[0], qmin1 = qb[1], qmin2 = qb[2];
        const uint32_t qmax0 = qb[3], qmax1 = qb[4], qmax2 = qb[5];
        const float hg = A.g_hmax ? (float)A.g_hmax[g] : 0.f;
        unsigned long long gstart = cursor;
        uint32_t cand_lane = 0;
        uint32_t fsize = 1;
        if (lane == 0) fa[0] = sysid;
        __syncwarp();
        while (fsize > 0) {
            uint32_t nsize = 0;
            // node records (and the cells' radii) one batch ahead, frontier
            // ids two batches ahead, so that no batch waits on a load that
            // depends on another load
            uint32_t node_nx = lane < fsize ? fa[lane] : 0u;
            uint32_t node_nx2 = lane + 32 < fsize ? fa[lane + 32] : 0u;
            uint4 rec_nx = make_uint4(0, 0, 0, 0);
            float hc_nx = 0.f;
            if (lane < fsize) {
                rec_nx = A.nd_walk[node_nx];
                if (A.mode >= 2) hc_nx = (float)A.nd_hmax[node_nx];
            }
            for (uint32_t base = 0; base < fsize; base += 32) {
                const uint32_t idx = base + lane;
                const bool act = idx < fsize;
                const uint32_t node = node_nx;
                const uint4 rec = rec_nx;
                const float hc = hc_nx;
                if (idx + 32 < fsize) {
                    node_nx = node_nx2;
                    rec_nx = A.nd_walk[node_nx];
                    if (A.mode >= 2) hc_nx = (float)A.nd_hmax[node_nx];
                }
                if (idx + 64 < fsize) node_nx2 = fa[idx + 64];
                bool emit = false;
                uint32_t nch = 0, child = 0;
                if (act) {
                    const int level = (int)((rec.x >> 21) & 31u);
                    const bool leaf = (rec.x >> 26) & 1u;
                    const uint32_t w = (1u << (kMaxLevel - level)) - 1u;
                    const uint32_t qx = rec.x & kQMax, qy = rec.y, qz = rec.z;
                    // gaps between [q, q + w + 1) and [qmin, qmax + 1) in grid units
                    const float gx = (float)max(0, max((int)qx - (int)(qmax0 + 1), (int)qmin0 - (int)(qx + w + 1)));
                    const float gy = (float)max(0, max((int)qy - (int)(qmax1 + 1), (int)qmin1 - (int)(qy + w + 1)));
                    const float gz = (float)max(0, max((int)qz - (int)(qmax2 + 1), (int)qmin2 - (int)(qz + w + 1)));
                    const float d2 = (gx * gx + gy * gy + gz * gz) * dq2;
                    const float R = short_bound(A.mode, A.r_fixed, hc, hg);
                    // margin: FP32 rounding of the bound and of the gaps
                    const bool near = d2 <= R * R * (1.0f + 64.0f * kU);
                    if (near) {
                        if (leaf) {
                            emit = true;
                            cand_lane += rec.w;
                        } else {
                            nch = rec.x >> 27;
                            child = rec.w;
                        }
                    }
                }
                const uint32_t emask = __ballot_sync(0xFFFFFFFFu, emit);
                const uint32_t k = __popc(emask);
                if (k) {
                    if (cursor + k > chunk_end) {
                        const unsigned long long sofar = cursor - gstart;
                        const unsigned long long want = 2 * (sofar + k) > kSChunk ? 2 * (sofar + k) : kSChunk;
                        unsigned long long nb = 0;
                        if (lane == 0) nb = atomicAdd(&st->pool_cursor, want);
                        nb = __shfl_sync(0xFFFFFFFFu, nb, 0);
                        if (!ovf && nb + want > A.cap_pool) {
                            if (lane == 0) atomicOr(&st->overflow, kOvfPool);
                            ovf = true;
                        }
                        if (!ovf) {
                            for (unsigned long long j = lane; j < sofar; j += 32) A.pool[nb + j] = A.pool[gstart + j];
                            __syncwarp();
                            gstart = nb;
                            cursor = nb + sofar;
                            chunk_end = nb + want;
                        } else {
                            chunk_end = ~0ull;
                        }
                    }
                    if (emit && !ovf) A.pool[cursor + __popc(emask & lt)] = node | kLeafTag;
                    cursor += k;
                }
                if (__ballot_sync(0xFFFFFFFFu, nch > 0u)) {  // deep in the tree most batches open none
                    uint32_t inc = nch;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const uint32_t tv = __shfl_up_sync(0xFFFFFFFFu, inc, off);
                        if (lane >= off) inc += tv;
                    }
                    const uint32_t tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
                    if (nsize + tot > F) {
                        if (lane == 0) atomicOr(&st->overflow, kOvfFrontier);
                        ovf = true;
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
        const uint32_t cand = __reduce_add_sync(0xFFFFFFFFu, cand_lane);
        const unsigned long long len = cursor - gstart;
        if (lane == 0) {
            A.g_off[g] = gstart;
            A.g_len[g] = (uint32_t)len;
            A.g_nepj[g] = cand;
        }
        acc_entries += len;
        acc_cand += cand;
    }
    if (lane == 0) {
        atomicAdd(&st->pool_needed, acc_entries);
        atomicAdd(&st->list_entries, acc_entries);
        atomicAdd(&st->n_epj, acc_cand);
    }
}

struct ShortPairArgs {
    DevState* st;
    const uint32_t* g_first;
    const uint32_t* g_count;
    const unsigned long long* g_off;
    const uint32_t* g_len;
    const uint32_t* pool;
    const uint32_t* nd_first;
    const uint32_t* nd_count;
    const float4* pf_hi;  // (x hi - c0, y, z, m)
    const float4* pf_lo;  // (x lo, y lo, z lo, eps^2)
    const double* x;      // FP64 positions in key order
    const double* y;
    const double* z;
    const double* h;      // cutoff radii in key order (null for the fixed type)
    const uint32_t* id;   // key order -> caller's row
    const uint32_t* sys;
    const SysBox* box;
    uint32_t* count;      // caller order
    double* rho;
    unsigned long long* info;  // neighbour pairs, candidate pairs, FP64 decisions
    int mode;
    double r_fixed;
};

// W(r, H) of the 3D Wendland C6 kernel; zero from q = r / H >= 1 on (the
// factor (1 - q)^8 clamped at zero, without a branch).
__device__ __forceinline__ float wendland_c6(float r, float invH) {
    const float q = r * invH;
    const float u = fmaxf(1.0f - q, 0.0f), u2 = u * u, u4 = u2 * u2, u8 = u4 * u4;
    const float poly = fmaf(q, fmaf(q, fmaf(q, 32.0f, 25.0f), 8.0f), 1.0f);
    return kWc6 * invH * invH * invH * u8 * poly;
}

// MODE is the cutoff type (FDPS_CUTOFF_*), fixed at compile time so that
// the pair loop carries no selection between them.
template <int MODE>
__global__ void __launch_bounds__(kSBlock, 8) k_short_pairs(ShortPairArgs A) {
    __shared__ float4 s_h[kSW][kSTile];
    __shared__ float4 s_l[kSW][kSTile];
    __shared__ float s_ih[kSW][kSTile];  // 1 / h_j (scatter and symmetric types)
    __shared__ uint32_t s_p[kSW][kSTile];
    __shared__ uint32_t s_first[kSW][32];
    __shared__ uint32_t s_start[kSW][32];
    DevState* st = A.st;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ngroups = (uint32_t)st->n_groups;
    unsigned long long n_pairs = 0, n_cand = 0, n_fb = 0;
    for (;;) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(&st->force_counter, 1u);
        g = __shfl_sync(0xFFFFFFFFu, g, 0);
        if (g >= ngroups) break;
        const uint32_t gf = A.g_first[g], ni = A.g_count[g];
        const unsigned long long off = A.g_off[g];
        const uint32_t len = A.g_len[g];
        const float L = (float)A.box[A.sys ? A.sys[gf] : 0u].L;
        const float Eabs = 1e-13f * L;  // error of the FP64 -> FP32 hi/lo parts
        // lanes: P i-slots x nsl slices of the candidates, so that small
        // groups keep the whole warp busy
        const uint32_t P = ni <= 16u ? ni : 32u;
        const uint32_t nsl = 32u / P;
        const uint32_t ip = lane % P, sl = lane / P;
        for (uint32_t ib = 0; ib < ni; ib += P) {
            const uint32_t i = ib + ip;
            const bool act = sl < nsl && i < ni;
            const uint32_t pi = gf + (act ? i : 0u);
            const float4 ih = A.pf_hi[pi], il = A.pf_lo[pi];
            const double hi64 = MODE != 0 ? A.h[pi] : A.r_fixed;
            const float hif = (float)hi64;
            const float invHi = 1.0f / (MODE == 0 ? (float)A.r_fixed : hif);
            // the cutoff of the fixed and gather types is the lane's own, and
            // so are two thresholds on r^2 that decide every pair the pair
            // bound below decides on the same side: M <= Mmax for r^2 <= c^2
            // (a <= r <= c), and for r^2 > c^2, with a <= r <= (r^2 + c^2) /
            // (2c), M <= (56u + 192u^2 + beta) r^2 + (8u + beta) c^2 + 3 Eabs^2,
            // beta = 3 Eabs / c (slack for the FP32 evaluation of both); a
            // cutoff within a few Eabs sends every pair to the FP64 sequence
            const float ci = MODE == 0 ? (float)A.r_fixed : hif, ci2 = ci * ci;
            float lo_thr = -INFINITY, hi_thr = INFINITY;
            if (MODE <= 1) {
                const float beta = 3.0001f * Eabs / ci;
                if (beta < 0.25f) {
                    const float tq = fmaf(8.0f * kU, ci, Eabs);
                    const float Mmax = 64.0f * kU * ci2 + 6.0f * ci * Eabs + 3.0f * tq * tq;
                    lo_thr = ci2 - (1.01f * Mmax + 4.0f * kU * ci2);
                    hi_thr = (ci2 * (1.0f + 8.0f * kU + beta) + 3.0f * Eabs * Eabs) * (1.0f + 16.0f * kU) /
                             (1.0f - (56.0f * kU + 192.0f * kU * kU + beta));
                }
            }
            uint32_t cnt = 0, cands = 0, fbk = 0;
            float sum = 0.0f;
            for (uint32_t base = 0; base < len; base += 32) {
                // leaves of this step: particle counts and offsets
                const uint32_t u = base + lane;
                const uint32_t node = u < len ? (A.pool[off + u] & ~kLeafTag) : 0u;
                const uint32_t c = u < len ? A.nd_count[node] : 0u;
                uint32_t inc = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t tv = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                    if (lane >= o) inc += tv;
                }
                const uint32_t total = __shfl_sync(0xFFFFFFFFu, inc, 31);
                __syncwarp();
                s_first[w][lane] = u < len ? A.nd_first[node] : 0u;
                s_start[w][lane] = inc - c;
                for (uint32_t c0 = 0; c0 < total; c0 += kSTile) {
                    const uint32_t m = total - c0 < (uint32_t)kSTile ? total - c0 : (uint32_t)kSTile;
                    __syncwarp();
                    for (uint32_t k = lane; k < m; k += 32) {
                        const uint32_t item = c0 + k;
                        int src = 0;
#pragma unroll
                        for (int step = 16; step > 0; step >>= 1)
                            if (s_start[w][src + step] <= item) src += step;
                        const uint32_t pj = s_first[w][src] + (item - s_start[w][src]);
                        const float4 lo = A.pf_lo[pj];
                        const float hj = MODE >= 2 ? (float)A.h[pj] : 0.0f;
                        s_h[w][k] = A.pf_hi[pj];
                        s_l[w][k] = make_float4(lo.x, lo.y, lo.z, hj);
                        if (MODE >= 2) s_ih[w][k] = 1.0f / hj;
                        s_p[w][k] = pj;
                    }
                    __syncwarp();
                    if (act) {
#pragma unroll 4
                        for (uint32_t k = sl; k < m; k += nsl) {
                            ++cands;
                            const float4 jh = s_h[w][k], jl = s_l[w][k];
                            const float dx = (jh.x - ih.x) + (jl.x - il.x);
                            const float dy = (jh.y - ih.y) + (jl.y - il.y);
                            const float dz = (jh.z - ih.z) + (jl.z - il.z);
                            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            bool near;  // inside the bound: the FP64 sequence decides
                            bool nb = false;
                            if (MODE <= 1) {
                                nb = r2 < lo_thr;
                                near = !nb && !(r2 > hi_thr);
                            } else {
                                const float c2 = MODE == 2 ? jl.w * jl.w : fmaxf(hif, jl.w) * fmaxf(hif, jl.w);
                                const float a = fmaxf(fmaxf(fabsf(dx), fabsf(dy)), fabsf(dz));
                                const float Ea = 8.0f * kU * a + Eabs;
                                const float M = 8.0f * kU * (r2 + c2) + 6.0f * a * Ea + 3.0f * Ea * Ea;
                                nb = r2 < c2 - M;
                                near = !nb && !(r2 > c2 + M);
                            }
                            if (near) {  // the exact FP64 sequence
                                ++fbk;
                                const uint32_t pj = s_p[w][k];
                                const double ex = __dsub_rn(A.x[pj], A.x[pi]);
                                const double ey = __dsub_rn(A.y[pj], A.y[pi]);
                                const double ez = __dsub_rn(A.z[pj], A.z[pi]);
                                const double e2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)),
                                                            __dmul_rn(ez, ez));
                                const double hj64 = MODE != 0 ? A.h[pj] : A.r_fixed;
                                const double cc = MODE == 0 ? A.r_fixed
                                                : MODE == 1 ? hi64
                                                : MODE == 2 ? hj64
                                                            : (hi64 > hj64 ? hi64 : hj64);
                                nb = e2 < __dmul_rn(cc, cc);
                            }
                            // the kernel for every candidate, kept for the
                            // neighbours only: a third of the pairs are
                            // neighbours, so a branch would be taken by some
                            // lane of nearly every step anyway
                            const float r = sqrtf(r2);
                            float wk;
                            if (MODE == 3)
                                wk = 0.5f * (wendland_c6(r, invHi) + wendland_c6(r, s_ih[w][k]));
                            else if (MODE == 2)
                                wk = wendland_c6(r, s_ih[w][k]);
                            else
                                wk = wendland_c6(r, invHi);
                            cnt += nb ? 1u : 0u;
                            sum = fmaf(jh.w, nb ? wk : 0.0f, sum);
                        }
                    }
                }
            }
            // the slices' partial counts and sums, into the first slice
            uint32_t cnt_all = cnt;
            float sum_all = sum;
            for (uint32_t q = 1; q < nsl; ++q) {
                const int src = (int)((ip + q * P) & 31u);
                cnt_all += __shfl_sync(0xFFFFFFFFu, cnt, src);
                sum_all += __shfl_sync(0xFFFFFFFFu, sum, src);
            }
            if (act && sl == 0) {
                const uint32_t row = A.id[pi];
                A.count[row] = cnt_all;
                A.rho[row] = (double)sum_all;
            }
            n_pairs += act ? cnt : 0u;
            n_cand += act ? cands : 0u;
            n_fb += act ? fbk : 0u;
        }
    }
    // per-warp totals
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_pairs += __shfl_xor_sync(0xFFFFFFFFu, n_pairs, o);
        n_cand += __shfl_xor_sync(0xFFFFFFFFu, n_cand, o);
        n_fb += __shfl_xor_sync(0xFFFFFFFFu, n_fb, o);
    }
    if (lane == 0 && A.info) {
        atomicAdd(&A.info[0], n_pairs);
        atomicAdd(&A.info[1], n_cand);
        atomicAdd(&A.info[2], n_fb);
    }
}

}  // namespace

int short_prepare(fdps_tree* t, fdps_psys* ps, int mode, const double* h_user) {
    fdps_ctx* ctx = t->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t n = ps->n;
    if (mode == 0) return FDPS_OK;  // the fixed cutoff needs no radii
    if (t->cap_sr_h < n) {
        dev_free(t->sr_h);
        t->cap_sr_h = 0;
        if (dev_alloc(&t->sr_h, n) != cudaSuccess) {
            cudaGetLastError();
            return set_error(ctx, FDPS_ENOMEM, "cutoff radii allocation failed");
        }
        t->cap_sr_h = n;
    }
    FDPS_CUDA_TRY(ctx, cudaMemsetAsync(ps->d_flag, 0, sizeof(uint32_t), s));
    k_short_h<<<grid_for(n, 256, 4 * ctx->sm_count), 256, 0, s>>>(n, ps->id[ps->cur], h_user, t->sr_h, ps->d_flag);
    FDPS_LAUNCH_CHECK(ctx);
    uint32_t bad = 0;
    FDPS_CUDA_TRY(ctx, cudaMemcpyAsync(&bad, ps->d_flag, sizeof(bad), cudaMemcpyDeviceToHost, s));
    FDPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (bad) return set_error(ctx, FDPS_EINVAL, "cutoff radii must be positive and finite");
    int rc = read_device_state(t);
    if (rc) return rc;
    const int64_t nn = t->h_st.n_nodes, ng = t->h_st.n_groups;
    if (t->cap_nd_hmax < nn) {
        dev_free(t->nd_hmax);
        t->cap_nd_hmax = 0;
        if (dev_alloc(&t->nd_hmax, t->cap_nodes) != cudaSuccess) {
            cudaGetLastError();
            return set_error(ctx, FDPS_ENOMEM, "node radii allocation failed");
        }
        t->cap_nd_hmax = t->cap_nodes;
    }
    if (t->cap_g_hmax < ng) {
        dev_free(t->g_hmax);
        t->cap_g_hmax = 0;
        if (dev_alloc(&t->g_hmax, t->cap_groups) != cudaSuccess) {
            cudaGetLastError();
            return set_error(ctx, FDPS_ENOMEM, "group radii allocation failed");
        }
        t->cap_g_hmax = t->cap_groups;
    }
    if (mode >= 2) {  // the cells' largest radii bound the j-dependent cutoffs only
        k_hmax_leaves<<<grid_for(nn, 256, 4 * ctx->sm_count), 256, 0, s>>>(nn, t->nd_meta, t->nd_first,
                                                                          t->nd_count, t->sr_h, t->nd_hmax);
        FDPS_LAUNCH_CHECK(ctx);
        for (int l = t->h_st.max_level - 1; l >= 0; --l) {
            const int64_t a = t->h_st.lvl_start[l], b = t->h_st.lvl_start[l + 1];
            if (b <= a) continue;
            k_hmax_internal<<<grid_for(b - a, 256, 4 * ctx->sm_count), 256, 0, s>>>(a, b, t->nd_meta,
                                                                                   t->nd_child, t->nd_hmax);
            FDPS_LAUNCH_CHECK(ctx);
        }
    }
    k_group_hmax<<<grid_for(ng, 256, 4 * ctx->sm_count), 256, 0, s>>>(ng, t->g_first, t->g_count, t->sr_h,
                                                                      t->g_hmax);
    FDPS_LAUNCH_CHECK(ctx);
    return FDPS_OK;
}

int launch_short_walk(fdps_tree* t, fdps_psys* ps, int mode, double r_fixed, int blocks) {
    fdps_ctx* ctx = t->ctx;
    ShortWalkArgs A;
    A.st = t->st;
    A.nd_walk = t->nd_walk;
    A.nd_hmax = mode >= 2 ? t->nd_hmax : nullptr;
    A.g_qbox = t->g_qbox;
    A.g_first = t->g_first;
    A.g_hmax = (mode == 1 || mode == 3) ? t->g_hmax : nullptr;
    A.sys = ps->d_sys;
    A.box = t->sys_box;
    A.g_off = t->g_off;
    A.g_len = t->g_len;
    A.g_nepj = t->g_nepj;
    A.pool = t->pool;
    A.cap_pool = (unsigned long long)t->cap_pool;
    A.frontier = t->frontier;
    A.cap_frontier = (uint32_t)t->cap_frontier;
    A.mode = mode;
    A.r_fixed = (float)r_fixed;
    k_short_walk<<<blocks, kSBlock, 0, ctx->stream>>>(A);
    FDPS_LAUNCH_CHECK(ctx);
    return FDPS_OK;
}

int launch_short_pairs(fdps_tree* t, fdps_psys* ps, int mode, double r_fixed, uint32_t* count, double* rho,
                       unsigned long long* info3) {
    fdps_ctx* ctx = t->ctx;
    const int c = ps->cur;
    ShortPairArgs A;
    A.st = t->st;
    A.g_first = t->g_first;
    A.g_count = t->g_count;
    A.g_off = t->g_off;
    A.g_len = t->g_len;
    A.pool = t->pool;
    A.nd_first = t->nd_first;
    A.nd_count = t->nd_count;
    A.pf_hi = t->pf_hi;
    A.pf_lo = t->pf_lo;
    A.x = ps->x[c];
    A.y = ps->y[c];
    A.z = ps->z[c];
    A.h = mode == 0 ? nullptr : t->sr_h;
    A.id = ps->id[c];
    A.sys = ps->d_sys;
    A.box = t->sys_box;
    A.count = count;
    A.rho = rho;
    A.info = info3;
    A.mode = mode;
    A.r_fixed = r_fixed;
    void (*kern)(ShortPairArgs) = mode == 0 ? k_short_pairs<0> : mode == 1 ? k_short_pairs<1>
                                : mode == 2 ? k_short_pairs<2> : k_short_pairs<3>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSBlock, 0) != cudaSuccess || per_sm < 1)
        per_sm = 4;
    kern<<<per_sm * ctx->sm_count, kSBlock, 0, ctx->stream>>>(A);
    FDPS_LAUNCH_CHECK(ctx);
    return FDPS_OK;
}

}  // namespace fdps
