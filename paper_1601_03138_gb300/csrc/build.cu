// build.cu -- octree build, bottom-up moments and i-groups.
//
// Octree (the Barnes-Hut tree of Sect. 3.2; its rules are this library's
// reading): a node is a (level l, key prefix) pair holding >= 1 particle; it
// is a leaf iff it holds <= n_leaf particles or l = 21; an internal node's
// children are its non-empty octants in digit order.  Node ids are BFS
// order: level-major, prefix ascending.  All levels are built at once from
// the sorted keys, one thread per position (see the particle-parallel build
// below).
//
// Moments: M and S = sum m x are accumulated in FP64 with explicitly
// rounded adds and multiplies (no FMA), leaves sequentially over their
// particles, internal nodes sequentially over their children in octant
// order; COM = S / M.  These fixed orders make the centres of mass, and
// thus the opening decisions of the walk, reproducible bit for bit.  The
// traceless quadrupole Q_ab = sum m (3 d_a d_b - |d|^2 delta_ab) about the
// COM (Sect. 2.1.2: FDPS ships superparticles up to the quadrupole) is summed over particles
// for leaves and combined from the children with the parallel-axis shift
// for internal nodes.
//
// i-groups (Barnes 1990; Sect. 5.5): the maximal nodes with <= n_grp
// particles, and leaves with more (possible only at level 21), in order of
// their first particle.
#include <algorithm>

#include "fdps_internal.cuh"

namespace fdps {
namespace {

constexpr int kB = 256;  // block size of the partitioned kernels

// Contiguous tile range [t0, t1) of block b when `ntile` tiles of kB items
// are split over gridDim.x blocks; the same split in every launch keeps the
// per-block partial sums consistent between the count and write kernels.
__device__ __forceinline__ void block_tiles(int64_t nitems, int64_t* t0, int64_t* t1) {
    int64_t ntile = (nitems + kB - 1) / kB;
    int64_t per = (ntile + gridDim.x - 1) / gridDim.x;
    *t0 = blockIdx.x * per;
    *t1 = *t0 + per < ntile ? *t0 + per : ntile;
}

__device__ __forceinline__ uint32_t block_sum(uint32_t v) {
    __shared__ uint32_t s[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
    if (lane == 0) s[w] = v;
    __syncthreads();
    uint32_t r = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += s[k];
    __syncthreads();
    return r;  // valid in thread 0
}

__device__ __forceinline__ uint32_t block_excl(uint32_t v, uint32_t* total) {
    __shared__ uint32_t s_w[33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        uint32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, off);
        if (lane >= off) inc += t;
    }
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (w == 0) {
        uint32_t t = lane < nw ? s_w[lane] : 0u;
        uint32_t ti = t;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t u = __shfl_up_sync(0xFFFFFFFFu, ti, off);
            if (lane >= off) ti += u;
        }
        if (lane < nw) s_w[lane] = ti - t;
        if (lane == nw - 1) s_w[32] = ti;
    }
    __syncthreads();
    uint32_t res = s_w[w] + inc - v;
    *total = s_w[32];
    __syncthreads();
    return res;
}

// Exclusive scan of part[0..np) in one block; returns the total in *tot.
__device__ void scan_partials(uint32_t* part, int np, uint32_t* tot) {
    const int per = (np + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per;
    uint32_t sum = 0;
    for (int k = 0; k < per; ++k)
        if (b + k < np) sum += part[b + k];
    uint32_t total;
    uint32_t off = block_excl(sum, &total);
    for (int k = 0; k < per; ++k)
        if (b + k < np) {
            uint32_t c = part[b + k];
            part[b + k] = off;
            off += c;
        }
    *tot = total;
}

__device__ __forceinline__ uint32_t meta_level(uint32_t m) { return m & 0xFFu; }
__device__ __forceinline__ uint32_t meta_nchild(uint32_t m) { return (m >> 8) & 0xFFu; }
__device__ __forceinline__ bool meta_leaf(uint32_t m) { return (m >> 16) & 1u; }

// Level 0: one root per system (node k = root of system k, owning
// positions off[k] .. off[k+1]; a single root over all n if off is null).
// The other levels' nodes come from the particle-parallel kernels below.
struct RootArgs {
    int n_roots;
    const int64_t* off;
    int64_t n;
    int n_leaf;
    uint32_t* nd_first;
    uint32_t* nd_count;
    uint32_t* nd_child;
    uint32_t* nd_meta;
    uint32_t* nd_parent;
    uint64_t* nd_qlo;
};

// (done by the blocks of the count pass, grid-strided)
__device__ __forceinline__ void write_roots(const RootArgs& R) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < R.n_roots;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = R.off ? R.off[k] : 0, b = R.off ? R.off[k + 1] : R.n;
        R.nd_first[k] = (uint32_t)a;
        R.nd_count[k] = (uint32_t)(b - a);
        R.nd_child[k] = 0xFFFFFFFFu;
        R.nd_meta[k] = (b - a <= R.n_leaf ? 1u : 0u) << 16;
        R.nd_parent[k] = 0xFFFFFFFFu;
        R.nd_qlo[k] = 0;
    }
}

// ------------------------------------------------ particle-parallel build
//
// All levels at once from the sorted keys.  D_j, the first level at which
// the keys of positions j-1 and j differ (0 where a system starts, 22 for
// equal keys), marks cell boundaries: the level-l cell holding position i
// runs from the last j <= i with D_j <= l to before the next j > i with
// D_j <= l (positions outside [0, n) count as D = 0).  Cells shrink with
// the level, so the leaf holding i is at LL_i, the first level whose cell
// holds <= n_leaf particles (21 if none), and every coarser cell holding i
// is an internal node.  Hence the nodes starting at i are levels
// max(D_i, 1) .. LL_i, and the nodes ending at j (holding j - 1, not j) are
// levels max(D_j, 1) .. LL_{j-1}.  Whether a cell holds <= n_leaf particles
// is decided within n_leaf <= 16 positions either side.  Node ids stay
// breadth-first (level-major, first particle ascending): id = start of the
// level + number of the level's nodes starting before i, from per-tile
// counts scanned per level and per-warp counts within the tile.

constexpr int kBT = 256;                    // threads per tile
constexpr int kBWarps = kBT / 32;
constexpr int kBRows = 8;                   // rows of 32 positions per warp
constexpr int kBSpan = 32 * kBRows;         // positions per warp
constexpr int kBTile = kBT * kBRows;        // positions per tile
constexpr int kHalo = kMaxLeaf;             // window either side of a row
static_assert(kBTile == kBuildTile && kBWarps == kBuildWarps, "tile shape shared with the allocation");
static_assert(kHalo == 16, "a row's window is 64 positions: 16 before, 32 own, 16 after");

__device__ __forceinline__ uint32_t first_diff_level(int64_t j, int64_t n, const uint64_t* __restrict__ keys,
                                                     const uint32_t* __restrict__ sys) {
    if (j <= 0 || j >= n) return 0u;
    if (sys && sys[j] != sys[j - 1]) return 0u;
    const uint64_t x = keys[j - 1] ^ keys[j];
    // keys have 63 bits: bit 62 is the top bit of the level-1 digit
    return x ? ((uint32_t)__clzll((long long)x) - 1u) / 3u + 1u : 22u;
}

// Does the cell holding window position c hold <= n_leaf particles, given
// the window's boundaries M (bit k: D of window position k <= the level)?
// A boundary missing on either side means more than 16 particles.
__device__ __forceinline__ bool cell_fits(unsigned long long M, int c, int n_leaf) {
    const unsigned long long back = M & ((2ull << c) - 1ull);
    const unsigned long long fwd = M >> (c + 1);
    if (!back || !fwd) return false;
    const int s = 63 - __clzll((long long)back);
    const int e = c + __ffsll((long long)fwd);
    return e - s <= n_leaf;
}

// Per tile: D and LL of every position (pk = D | LL << 8) and the number of
// nodes of each level starting in each warp's positions, per warp
// (wcount[(l - 1) * nw + warp]) and per tile (tcount[(l - 1) * ntiles +
// tile]).  A warp takes 32 consecutive positions at a time: 22 ballots give
// each level's boundaries in the 64-position window around them, and each
// lane bisects the levels for its LL.
__global__ void __launch_bounds__(kBT) k_tree_count(int64_t n, int n_leaf, const uint64_t* __restrict__ keys,
                                                    const uint32_t* __restrict__ sys, uint32_t* __restrict__ pk,
                                                    uint32_t* __restrict__ wcount, uint32_t* __restrict__ tcount,
                                                    int64_t nw, int64_t ntiles, RootArgs R) {
    write_roots(R);  // level 0 (no other work of this pass depends on it)
    __shared__ uint8_t sD[kBTile + 2 * kHalo];
    __shared__ unsigned long long s_m[kBWarps][kMaxLevel + 1];
    __shared__ uint32_t s_wc[kMaxLevel][kBWarps];
    const int64_t t0 = (int64_t)blockIdx.x * kBTile;
    for (int q = threadIdx.x; q < kBTile + 2 * kHalo; q += kBT)
        sD[q] = (uint8_t)first_diff_level(t0 - kHalo + q, n, keys, sys);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = kHalo + lane;  // own window position
    uint32_t cnt[kMaxLevel];
#pragma unroll
    for (int l = 0; l < kMaxLevel; ++l) cnt[l] = 0u;
    for (int r = 0; r < kBRows; ++r) {
        const int rb = w * kBSpan + r * 32;  // tile position of the row's first position
        const int64_t i = t0 + rb + lane;
        const uint32_t dA = sD[rb + lane];       // window 0..31
        const uint32_t dB = sD[rb + 32 + lane];  // window 32..63
        const uint32_t d = sD[rb + kHalo + lane];
#pragma unroll
        for (int l = 0; l <= kMaxLevel; ++l) {
            const uint32_t a = __ballot_sync(0xFFFFFFFFu, dA <= (uint32_t)l);
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, dB <= (uint32_t)l);
            if (lane == 0) s_m[w][l] = (unsigned long long)a | ((unsigned long long)b << 32);
        }
        __syncwarp();
        int lo = 0, hi = kMaxLevel;  // first fitting level in [lo, hi], or 21
#pragma unroll
        for (int it = 0; it < 5; ++it) {
            const int mid = (lo + hi) >> 1;
            if (lo < hi) {
                if (cell_fits(s_m[w][mid], c, n_leaf))
                    hi = mid;
                else
                    lo = mid + 1;
            }
        }
        const uint32_t LL = (uint32_t)lo;
        __syncwarp();  // s_m is rewritten by the next row
        if (i < n) pk[i] = d | (LL << 8);
        const uint32_t l0 = max(d, 1u);
        const uint32_t mask = (i < n && l0 <= LL) ? ((2u << LL) - (1u << l0)) : 0u;
#pragma unroll
        for (int l = 1; l <= kMaxLevel; ++l) cnt[l - 1] += __popc(__ballot_sync(0xFFFFFFFFu, (mask >> l) & 1u));
    }
    uint32_t mine = 0u;
#pragma unroll
    for (int l = 0; l < kMaxLevel; ++l)
        if (lane == l) mine = cnt[l];
    if (lane < kMaxLevel) {
        wcount[(int64_t)lane * nw + (int64_t)blockIdx.x * kBWarps + w] = mine;
        s_wc[lane][w] = mine;
    }
    __syncthreads();
    if (threadIdx.x < kMaxLevel) {
        uint32_t t = 0u;
#pragma unroll
        for (int k = 0; k < kBWarps; ++k) t += s_wc[threadIdx.x][k];
        tcount[(int64_t)threadIdx.x * ntiles + blockIdx.x] = t;
    }
}

// Exclusive scan of one level's per-tile counts (block l - 1 takes level
// l); the level's total goes to ltot[l - 1].
__global__ void __launch_bounds__(1024) k_tree_scan(uint32_t* tcount, int64_t ntiles, uint32_t* ltot) {
    uint32_t tot;
    scan_partials(tcount + (int64_t)blockIdx.x * ntiles, (int)ntiles, &tot);
    if (threadIdx.x == 0) ltot[blockIdx.x] = tot;
}

__device__ __forceinline__ uint32_t compact3(uint64_t v) {
    v &= 0x1249249249249249ull;
    v = (v | (v >> 2)) & 0x10C30C30C30C30C3ull;
    v = (v | (v >> 4)) & 0x100F00F00F00F00Full;
    v = (v | (v >> 8)) & 0x001F0000FF0000FFull;
    v = (v | (v >> 16)) & 0x001F00000000FFFFull;
    v = (v | (v >> 32)) & 0x1FFFFFull;
    return (uint32_t)v;
}

// Writes every node of levels >= 1: first particle, level and leaf flag,
// parent, first child, grid origin, and (in nd_count, turned into the
// count by k_tree_finish) the position after its last particle.  The
// level-l node holding j - 1 is the last level-l node that starts before j,
// so a position's exclusive rank at each level names both the nodes it
// starts and those it ends.  The blocks cover positions 0 .. n (every open
// node ends at n).  Each block derives the level starts from the totals
// (levels from the first that does not fit in the node arrays on are left
// empty, with the overflow flag set); block 0 also publishes them.
__global__ void __launch_bounds__(kBT) k_tree_nodes(
    int64_t n, int n_roots, int64_t cap_nodes, const uint64_t* __restrict__ keys,
    const uint32_t* __restrict__ sys, const uint32_t* __restrict__ pk, const uint32_t* __restrict__ wcount,
    const uint32_t* __restrict__ tcount, int64_t nw, int64_t ntiles, const uint32_t* __restrict__ ltot,
    DevState* st, uint32_t* __restrict__ nd_first, uint32_t* __restrict__ nd_end, uint32_t* __restrict__ nd_child,
    uint32_t* __restrict__ nd_meta, uint32_t* __restrict__ nd_parent, uint64_t* __restrict__ nd_qlo) {
    __shared__ int64_t s_lvl[kMaxLevel + 3];
    __shared__ int s_cut;
    __shared__ uint32_t s_wc[kMaxLevel][kBWarps];
    __shared__ uint32_t sP[1 + kBTile];  // pk of positions t0 - 1 .. t0 + kBTile - 1
    if (threadIdx.x == 0) {
        int64_t s = n_roots;
        // keys left unsorted by a sort that gave up: roots only, so that
        // every later stage stays within its buffers until the retry
        const bool stalled = st->overflow & kSortInvalid;
        int cut = stalled ? 1 : kMaxLevel + 1, top = 0;
        s_lvl[0] = 0;
        for (int l = 1; l <= kMaxLevel; ++l) {
            s_lvl[l] = s;
            if (cut > kMaxLevel && s + ltot[l - 1] > cap_nodes) cut = l;
            if (cut > kMaxLevel) {
                s += ltot[l - 1];
                if (ltot[l - 1]) top = l;
            }
        }
        for (int l = cut; l <= kMaxLevel + 2; ++l) s_lvl[l] = s;
        s_cut = cut;
        if (blockIdx.x == 0) {
            for (int l = 0; l < kMaxLevel + 3; ++l) st->lvl_start[l] = (int32_t)s_lvl[l];
            st->n_nodes = (int32_t)s;
            st->max_level = top;
            if (cut <= kMaxLevel && !stalled) st->overflow |= kOvfNodes;
        }
    }
    const int64_t tile = blockIdx.x;
    const int64_t t0 = tile * kBTile;
    // positions at or past n: D = 0, no nodes
    for (int q = threadIdx.x; q < 1 + kBTile; q += kBT) {
        const int64_t j = t0 - 1 + q;
        sP[q] = (j >= 0 && j < n) ? pk[j] : 0u;
    }
    if (threadIdx.x < kMaxLevel * kBWarps) {
        const int l = threadIdx.x / kBWarps, k = threadIdx.x % kBWarps;
        s_wc[l][k] = tile < ntiles ? wcount[(int64_t)l * nw + tile * kBWarps + k] : 0u;
    }
    __syncthreads();
    const int cut = s_cut;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    // next id of each level for this warp: level start + nodes of earlier
    // tiles + nodes of earlier warps of this tile (a tile past the counted
    // ones holds only position n: all of the level's nodes come before)
    uint32_t nxt = 0u;
    if (lane >= 1 && lane <= kMaxLevel) {
        nxt = (uint32_t)s_lvl[lane] + (tile < ntiles ? tcount[(int64_t)(lane - 1) * ntiles + tile] : ltot[lane - 1]);
        for (int k = 0; k < w; ++k) nxt += s_wc[lane - 1][k];
    }
    uint32_t run[kMaxLevel];
#pragma unroll
    for (int l = 1; l <= kMaxLevel; ++l) run[l - 1] = __shfl_sync(0xFFFFFFFFu, nxt, l);
    for (int r = 0; r < kBRows; ++r) {
        const int p = w * kBSpan + r * 32 + lane;
        const int64_t j = t0 + p;
        const uint32_t v = sP[1 + p], u = sP[p];
        const uint32_t d = v & 0xFFu, LL = (v >> 8) & 0xFFu;
        const uint32_t lo = max(d, 1u), hi = LL;
        const bool any = j < n && lo <= hi;
        // levels of the nodes that end here
        uint32_t elo = 32u, ehi = 0u;
        if (j >= 1 && j <= n && d <= (uint32_t)kMaxLevel) {
            elo = max(d, 1u);
            ehi = (u >> 8) & 0xFFu;
        }
        uint64_t key = 0;
        uint32_t qx = 0, qy = 0, qz = 0, root = 0;
        if (any) {
            key = keys[j];
            qx = compact3(key >> 2);
            qy = compact3(key >> 1);
            qz = compact3(key);
            if (sys) root = sys[j];
        }
        uint32_t prev_id = 0u, prev_excl = 0u;
#pragma unroll
        for (int l = 1; l <= kMaxLevel; ++l) {
            const bool h = any && lo <= (uint32_t)l && (uint32_t)l <= hi;
            const uint32_t bm = __ballot_sync(0xFFFFFFFFu, h);
            const uint32_t excl = run[l - 1] + __popc(bm & lt);
            run[l - 1] += __popc(bm);
            if (l < cut) {
                if (elo <= (uint32_t)l && (uint32_t)l <= ehi) nd_end[excl - 1u] = (uint32_t)j;
                if (h) {
                    const uint32_t id = excl;
                    uint32_t parent;
                    if ((uint32_t)l > lo) {
                        parent = prev_id;
                        nd_child[prev_id] = id;  // first child of this position's previous node
                    } else if (l == 1) {
                        parent = root;
                        if (d == 0u) nd_child[root] = id;  // a system's first position
                    } else {
                        parent = prev_excl - 1u;  // last node of level l - 1 starting before j
                    }
                    const uint32_t cm = ~((1u << (kMaxLevel - l)) - 1u) & kQMax;
                    nd_first[id] = (uint32_t)j;
                    nd_child[id] = 0xFFFFFFFFu;
                    nd_meta[id] = (uint32_t)l | (((uint32_t)l == hi ? 1u : 0u) << 16);
                    nd_parent[id] = parent;
                    nd_qlo[id] = ((uint64_t)(qx & cm) << 42) | ((uint64_t)(qy & cm) << 21) | (uint64_t)(qz & cm);
                    prev_id = id;
                }
            }
            prev_excl = excl;
        }
    }
}

// Counts (end - first) and children counts: node c is the last child of
// its parent P iff the next node has another parent; it then stores c -
// first child of P + 1 in P's meta (one writer per parent).
__global__ void __launch_bounds__(256) k_tree_finish(const DevState* __restrict__ st, int n_roots,
                                                     const uint32_t* __restrict__ nd_first,
                                                     uint32_t* __restrict__ nd_count,
                                                     const uint32_t* __restrict__ nd_parent,
                                                     const uint32_t* __restrict__ nd_child,
                                                     uint32_t* __restrict__ nd_meta) {
    const int64_t nn = st->n_nodes;
    for (int64_t c = n_roots + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nn;
         c += (int64_t)gridDim.x * blockDim.x) {
        nd_count[c] -= nd_first[c];
        const uint32_t P = nd_parent[c];
        if (c + 1 == nn || nd_parent[c + 1] != P) nd_meta[P] |= ((uint32_t)c - nd_child[P] + 1u) << 8;
    }
}

// ------------------------------------------------------------ moments

__device__ __forceinline__ void split_hilo(double v, float* hi, float* lo) { split_f32(v, *hi, *lo); }

// S / M correctly rounded.  With one reciprocal y = RN(1/M) for a node's three
// quotients, Markstein's correction q0 = RN(S y), r = RN(S - M q0) and
// q = RN(q0 + r y), each step one fused multiply-add, gives RN(S / M)
// (Markstein 1990); the exponent guards keep every intermediate a normal
// number, elsewhere the division instruction sequence runs.
__device__ __forceinline__ bool exp_mid(double v) {
    const int e = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
    return e >= 200 && e <= 1850;
}
__device__ __forceinline__ double quot(double S, double M, double y, bool ok) {
    if (!ok || !exp_mid(S)) return __ddiv_rn(S, M);  // zero, tiny or huge S: the division
    const double q0 = __dmul_rn(S, y);
    return __fma_rn(__fma_rn(-M, q0, S), y, q0);
}

struct MomArgs {
    const DevState* st;
    const SysBox* box;
    const uint32_t* sys;
    const double* px;
    const double* py;
    const double* pz;
    const double* pm;
    const double* pmx;  // m x, m y, m z per particle, each product rounded once
    const double* pmy;
    const double* pmz;
    const float4* pf_hi;
    const float4* pf_lo;
    const uint32_t* nd_first;
    const uint32_t* nd_count;
    const uint32_t* nd_child;
    const uint32_t* nd_meta;
    const uint32_t* nd_parent;
    const uint64_t* nd_qlo;
    // written here and read back for the parent in a later launch (read
    // through L2 with __ldcg)
    double* nd_sx;
    double* nd_sy;
    double* nd_sz;
    dvec4* nd_com;
    double* nd_quad;
    float4* nd_f;
    uint4* nd_walk;
    float4* nd_fq0;
    float2* nd_fq1;
};

// Moments of node i, whose children (if any) are complete.  M and S = sum
// m x in FP64 with every operation rounded on its own: leaves sequentially
// over their particles (the products m x come rounded from the reorder,
// where every lane has a particle; a lane here sums one leaf of up to
// n_leaf particles, so its multiplications would idle the lanes of the
// warp's smaller leaves on the narrow FP64 pipe), internal nodes over their
// children in octant order.  Quadrupole: FP64 (Q64) for the FP64 pipeline; otherwise FP32 from
// positions relative to the node's COM formed from FP32 hi/lo pairs, and the
// parallel-axis shift for internal nodes.
template <bool QUAD, bool Q64>
__device__ __forceinline__ void node_moments(const MomArgs& A, int64_t i) {
    const uint32_t meta = A.nd_meta[i];
    const bool leaf = meta_leaf(meta);
    const uint32_t f = A.nd_first[i], cnt = A.nd_count[i];
    const uint32_t c0 = A.nd_child[i], nc = meta_nchild(meta);
    const SysBox& bx = A.box[A.sys ? A.sys[f] : 0];
    double M = 0.0, Sx = 0.0, Sy = 0.0, Sz = 0.0;
    if (leaf) {
        for (uint32_t p = f; p < f + cnt; ++p) {
            M = __dadd_rn(M, A.pm[p]);
            Sx = __dadd_rn(Sx, A.pmx[p]);
            Sy = __dadd_rn(Sy, A.pmy[p]);
            Sz = __dadd_rn(Sz, A.pmz[p]);
        }
    } else {
        for (uint32_t c = c0; c < c0 + nc; ++c) {
            M = __dadd_rn(M, __ldcg(&A.nd_com[c].w));
            Sx = __dadd_rn(Sx, __ldcg(&A.nd_sx[c]));
            Sy = __dadd_rn(Sy, __ldcg(&A.nd_sy[c]));
            Sz = __dadd_rn(Sz, __ldcg(&A.nd_sz[c]));
        }
    }
    double cx = 0.0, cy = 0.0, cz = 0.0;
    if (M > 0.0) {
        const bool ok = exp_mid(M);
        const double y = ok ? __ddiv_rn(1.0, M) : 0.0;
        cx = quot(Sx, M, y, ok);
        cy = quot(Sy, M, y, ok);
        cz = quot(Sz, M, y, ok);
    }
    A.nd_sx[i] = Sx;
    A.nd_sy[i] = Sy;
    A.nd_sz[i] = Sz;
    A.nd_com[i] = make_dvec4(cx, cy, cz, M);
    float hx, hy, hz, lx, ly, lz;
    split_hilo(cx - bx.c0[0], &hx, &lx);
    split_hilo(cy - bx.c0[1], &hy, &ly);
    split_hilo(cz - bx.c0[2], &hz, &lz);
    A.nd_f[2 * i] = make_float4(hx, hy, hz, to_f32(M));
    A.nd_f[2 * i + 1] = make_float4(lx, ly, lz, 0.0f);
    // walk record: (q_x | level << 21 | leaf << 26 | children << 27, q_y, q_z,
    // first child of an internal node or particle count of a leaf)
    const uint64_t qlo = A.nd_qlo[i];
    const uint32_t lev = meta_level(meta), nch = nc;
    A.nd_walk[i] = make_uint4((uint32_t)(qlo >> 42) | (lev << 21) | ((leaf ? 1u : 0u) << 26) | (nch << 27),
                              (uint32_t)(qlo >> 21) & kQMax, (uint32_t)qlo & kQMax, leaf ? cnt : c0);
    if (!QUAD) return;
    if (Q64) {
        double q[6] = {0, 0, 0, 0, 0, 0};
        if (leaf) {
            for (uint32_t p = f; p < f + cnt; ++p) {
                const double m = A.pm[p];
                const double dx = A.px[p] - cx, dy = A.py[p] - cy, dz = A.pz[p] - cz;
                const double d2 = dx * dx + dy * dy + dz * dz;
                q[0] += m * (3.0 * dx * dx - d2);
                q[1] += m * (3.0 * dy * dy - d2);
                q[2] += m * (3.0 * dz * dz - d2);
                q[3] += m * (3.0 * dx * dy);
                q[4] += m * (3.0 * dx * dz);
                q[5] += m * (3.0 * dy * dz);
            }
        } else {
            for (uint32_t c = c0; c < c0 + nc; ++c) {
                const double ccx = __ldcg(&A.nd_com[c].x), ccy = __ldcg(&A.nd_com[c].y),
                             ccz = __ldcg(&A.nd_com[c].z), ccm = __ldcg(&A.nd_com[c].w);
                const double dx = ccx - cx, dy = ccy - cy, dz = ccz - cz;
                const double d2 = dx * dx + dy * dy + dz * dz;
                const double* qc = A.nd_quad + 6 * (int64_t)c;
                q[0] += __ldcg(qc + 0) + ccm * (3.0 * dx * dx - d2);
                q[1] += __ldcg(qc + 1) + ccm * (3.0 * dy * dy - d2);
                q[2] += __ldcg(qc + 2) + ccm * (3.0 * dz * dz - d2);
                q[3] += __ldcg(qc + 3) + ccm * (3.0 * dx * dy);
                q[4] += __ldcg(qc + 4) + ccm * (3.0 * dx * dz);
                q[5] += __ldcg(qc + 5) + ccm * (3.0 * dy * dz);
            }
        }
        double* qo = A.nd_quad + 6 * i;
#pragma unroll
        for (int k = 0; k < 6; ++k) qo[k] = q[k];
        A.nd_fq0[i] = make_float4((float)q[0], (float)q[1], (float)q[2], (float)q[3]);
        A.nd_fq1[i] = make_float2((float)q[4], (float)q[5]);
    } else {
        float q[6] = {0, 0, 0, 0, 0, 0};
        if (leaf) {
            for (uint32_t p = f; p < f + cnt; ++p) {
                const float4 ph = A.pf_hi[p], pl = A.pf_lo[p];
                const float m = ph.w;
                const float dx = (ph.x - hx) + (pl.x - lx), dy = (ph.y - hy) + (pl.y - ly),
                            dz = (ph.z - hz) + (pl.z - lz);
                const float d2 = dx * dx + dy * dy + dz * dz;
                q[0] += m * (3.0f * dx * dx - d2);
                q[1] += m * (3.0f * dy * dy - d2);
                q[2] += m * (3.0f * dz * dz - d2);
                q[3] += m * (3.0f * dx * dy);
                q[4] += m * (3.0f * dx * dz);
                q[5] += m * (3.0f * dy * dz);
            }
        } else {
            for (uint32_t c = c0; c < c0 + nc; ++c) {
                const float4 ch = __ldcg(&A.nd_f[2 * c]), cl = __ldcg(&A.nd_f[2 * c + 1]);
                const float4 q0 = __ldcg(&A.nd_fq0[c]);
                const float2 q1 = __ldcg(&A.nd_fq1[c]);
                const float dx = (ch.x - hx) + (cl.x - lx), dy = (ch.y - hy) + (cl.y - ly),
                            dz = (ch.z - hz) + (cl.z - lz);
                const float d2 = dx * dx + dy * dy + dz * dz;
                const float m = ch.w;
                q[0] += q0.x + m * (3.0f * dx * dx - d2);
                q[1] += q0.y + m * (3.0f * dy * dy - d2);
                q[2] += q0.z + m * (3.0f * dz * dz - d2);
                q[3] += q0.w + m * (3.0f * dx * dy);
                q[4] += q1.x + m * (3.0f * dx * dz);
                q[5] += q1.y + m * (3.0f * dy * dz);
            }
        }
        A.nd_fq0[i] = make_float4(q[0], q[1], q[2], q[3]);
        A.nd_fq1[i] = make_float2(q[4], q[5]);
    }
}

// Systems of an ensemble with at most this many particles get their whole
// subtree from one CTA (k_moments_systems); larger ones, and a single
// system, go through the leaf pass and one pass per level.
constexpr int64_t kSysMomMax = int64_t(1) << 17;

// Does the level-by-level pass skip node i (its system is done by
// k_moments_systems)?
__device__ __forceinline__ bool small_system_node(const MomArgs& A, const int64_t* off, int64_t i) {
    if (!off) return false;
    const uint32_t s = A.sys[A.nd_first[i]];
    return off[s + 1] - off[s] <= kSysMomMax;
}

// Leaves (of every level) in one launch, then the internal nodes level by
// level from the deepest up: each internal node finds its children complete.
template <bool QUAD, bool Q64>
__global__ void __launch_bounds__(256) k_moments_leaves(MomArgs A, const int64_t* off) {
    const int64_t nn = A.st->n_nodes;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
         i += (int64_t)gridDim.x * blockDim.x)
        if (meta_leaf(A.nd_meta[i]) && !small_system_node(A, off, i)) node_moments<QUAD, Q64>(A, i);
}

template <bool QUAD, bool Q64>
__global__ void __launch_bounds__(256) k_moments_internal(MomArgs A, const int64_t* off, int l) {
    const int64_t a = A.st->lvl_start[l], b = A.st->lvl_start[l + 1];
    for (int64_t i = a + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!meta_leaf(A.nd_meta[i]) && !small_system_node(A, off, i)) node_moments<QUAD, Q64>(A, i);
}

// First node of level range [lo, hi) whose first particle is >= p (the
// nodes of a level are ordered by their first particle).
__device__ __forceinline__ int64_t level_lower_bound(const uint32_t* nd_first, int64_t lo, int64_t hi, int64_t p) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)nd_first[mid] < p)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// One CTA per system of at most kSysMomMax particles (systems taken from a
// counter, largest first): the system's nodes level by level from the deepest up, with the
// same per-node code as the level passes, so the sums (and the centres of
// mass) come out bit for bit the same; one launch instead of 22.
template <bool QUAD, bool Q64>
__global__ void __launch_bounds__(256) k_moments_systems(MomArgs A, const int64_t* __restrict__ off,
                                                       const int32_t* __restrict__ order, int32_t n_sys,
                                                       uint32_t* counter) {
    __shared__ int32_t s_k;
    __shared__ int64_t s_rng[2 * (kMaxLevel + 1)];
    for (;;) {
        if (threadIdx.x == 0) s_k = (int32_t)atomicAdd(counter, 1u);
        __syncthreads();
        if (s_k >= n_sys) break;
        const int32_t k = order[s_k];  // largest systems first
        const int64_t a = off[k], b = off[k + 1];
        if (b - a <= kSysMomMax) {
            if (threadIdx.x <= kMaxLevel) {
                const int l = threadIdx.x;
                const int64_t lo = A.st->lvl_start[l], hi = A.st->lvl_start[l + 1];
                s_rng[2 * l] = level_lower_bound(A.nd_first, lo, hi, a);
                s_rng[2 * l + 1] = level_lower_bound(A.nd_first, lo, hi, b);
            }
            __syncthreads();
            for (int l = kMaxLevel; l >= 0; --l) {
                for (int64_t i = s_rng[2 * l] + threadIdx.x; i < s_rng[2 * l + 1]; i += blockDim.x)
                    node_moments<QUAD, Q64>(A, i);
                __syncthreads();  // this level complete before its parents
            }
        }
        __syncthreads();  // s_k and s_rng are rewritten next round
    }
}

template <bool QUAD, bool Q64>
int launch_moments(fdps_ctx* ctx, const MomArgs& A, const fdps_psys* ps, DevState* st) {
    const int grid = ctx->sm_count * 8;
    const int64_t* off = ps->n_sys > 1 ? ps->d_off : nullptr;
    if (off) {
        const int g = (int)std::min<int64_t>(ps->n_sys, (int64_t)ctx->sm_count * 8);
        k_moments_systems<QUAD, Q64><<<g, 256, 0, ctx->stream>>>(A, off, ps->d_order, ps->n_sys, &st->mom_counter);
        FDPS_LAUNCH_CHECK(ctx);
        if (ps->max_sys_n <= kSysMomMax) return FDPS_OK;
    }
    k_moments_leaves<QUAD, Q64><<<grid, 256, 0, ctx->stream>>>(A, off);
    FDPS_LAUNCH_CHECK(ctx);
    for (int l = kMaxLevel - 1; l >= 0; --l) {
        k_moments_internal<QUAD, Q64><<<grid, 256, 0, ctx->stream>>>(A, off, l);
        FDPS_LAUNCH_CHECK(ctx);
    }
    return FDPS_OK;
}

// ------------------------------------------------------------- groups

__global__ void __launch_bounds__(256) k_group_mark(const DevState* __restrict__ st, int n_grp,
                                                    int n_roots,
                                                    const uint32_t* __restrict__ nd_first,
                                                    const uint32_t* __restrict__ nd_count,
                                                    const uint32_t* __restrict__ nd_meta,
                                                    const uint32_t* __restrict__ nd_parent,
                                                    uint32_t* __restrict__ head) {
    const int64_t nn = st->n_nodes;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = nd_count[i];
        const bool cand = c <= (uint32_t)n_grp || meta_leaf(nd_meta[i]);
        if (cand && (i < n_roots || nd_count[nd_parent[i]] > (uint32_t)n_grp)) head[nd_first[i]] = (uint32_t)i;
    }
}

// Group heads per block; the last block to finish (counted in
// st->grp_done, zero on entry) scans the per-block counts into offsets and
// publishes the number of groups.
__global__ void __launch_bounds__(kB) k_group_count(int64_t n, const uint32_t* __restrict__ head,
                                                    uint32_t* __restrict__ part, DevState* st,
                                                    int64_t cap_groups) {
    __shared__ bool s_last;
    int64_t t0, t1;
    block_tiles(n, &t0, &t1);
    uint32_t c = 0;
    for (int64_t t = t0; t < t1; ++t) {
        const int64_t i = t * kB + threadIdx.x;
        if (i < n && head[i] != 0xFFFFFFFFu) ++c;
    }
    uint32_t tot = block_sum(c);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = tot;
        __threadfence();  // the count is visible before the block counts itself done
        s_last = atomicAdd(&st->grp_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int np = (int)gridDim.x;
    const int per = (np + kB - 1) / kB;
    const int b = threadIdx.x * per;
    uint32_t sum = 0;
    for (int k = 0; k < per; ++k)
        if (b + k < np) sum += __ldcg(&part[b + k]);
    uint32_t total;
    uint32_t off = block_excl(sum, &total);
    for (int k = 0; k < per; ++k)
        if (b + k < np) {
            const uint32_t v = __ldcg(&part[b + k]);
            part[b + k] = off;
            off += v;
        }
    if (threadIdx.x == 0) {
        if ((int64_t)total > cap_groups) st->overflow |= kOvfGroups;
        st->n_groups = (int32_t)((int64_t)total > cap_groups ? cap_groups : total);
    }
}

__global__ void __launch_bounds__(kB) k_group_write(int64_t n, int64_t cap_groups,
                                                    const uint32_t* __restrict__ head,
                                                    const uint32_t* __restrict__ part,
                                                    const uint32_t* __restrict__ nd_count,
                                                    uint32_t* __restrict__ g_node,
                                                    uint32_t* __restrict__ g_first,
                                                    uint32_t* __restrict__ g_count) {
    int64_t t0, t1;
    block_tiles(n, &t0, &t1);
    uint32_t running = part[blockIdx.x];
    for (int64_t t = t0; t < t1; ++t) {
        const int64_t i = t * kB + threadIdx.x;
        const uint32_t h = i < n ? head[i] : 0xFFFFFFFFu;
        const uint32_t flag = h != 0xFFFFFFFFu ? 1u : 0u;
        uint32_t tot;
        const uint32_t rank = block_excl(flag, &tot);
        if (flag) {
            const int64_t g = (int64_t)running + rank;
            if (g < cap_groups) {
                g_node[g] = h;
                g_first[g] = (uint32_t)i;
                g_count[g] = nd_count[h];
            }
        }
        running += tot;
    }
}

__device__ __forceinline__ unsigned long long ord64(double v) {
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double unord64(unsigned long long o) {
    unsigned long long u = (o >> 63) ? (o & 0x7FFFFFFFFFFFFFFFull) : ~o;
    return __longlong_as_double((long long)u);
}

// FP64 box of each group (min / max over its particles), its grid box (the
// quantised corners: quantisation is monotone, so these are the minimum and
// maximum grid coordinates of the particles), FP64 centre and the FP32
// copies the walk's filter and the force kernel use.  A warp takes 32
// groups: the lanes reduce each group's particles together, then every lane
// finishes one group's FP64 arithmetic.
__global__ void __launch_bounds__(256) k_group_data(
    const DevState* __restrict__ st, const SysBox* __restrict__ box, const uint32_t* __restrict__ sys,
    const uint32_t* __restrict__ g_first,
    const uint32_t* __restrict__ g_count, const double* __restrict__ px,
    const double* __restrict__ py, const double* __restrict__ pz, double* __restrict__ g_box,
    uint32_t* __restrict__ g_qbox, dvec4* __restrict__ g_c64, float4* __restrict__ g_ch,
    float4* __restrict__ g_cl, float4* __restrict__ g_blo, float4* __restrict__ g_bhi) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t ng = st->n_groups;
    for (int64_t base = warp * 32; base < ng; base += nwarps * 32) {
        unsigned long long mlo[3] = {0, 0, 0}, mhi[3] = {0, 0, 0};
        const int nb = ng - base < 32 ? (int)(ng - base) : 32;
        for (int j = 0; j < nb; ++j) {
            const uint32_t f = g_first[base + j], c = g_count[base + j];
            unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
            for (uint32_t p = f + lane; p < f + c; p += 32) {
                unsigned long long v[3] = {ord64(px[p]), ord64(py[p]), ord64(pz[p])};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    lo[a] = v[a] < lo[a] ? v[a] : lo[a];
                    hi[a] = v[a] > hi[a] ? v[a] : hi[a];
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    unsigned long long l2 = __shfl_xor_sync(0xFFFFFFFFu, lo[a], off);
                    unsigned long long h2 = __shfl_xor_sync(0xFFFFFFFFu, hi[a], off);
                    lo[a] = l2 < lo[a] ? l2 : lo[a];
                    hi[a] = h2 > hi[a] ? h2 : hi[a];
                }
            if (lane == j)
                for (int a = 0; a < 3; ++a) {
                    mlo[a] = lo[a];
                    mhi[a] = hi[a];
                }
        }
        if (lane >= nb) continue;
        const int64_t g = base + lane;
        const SysBox& bx = box[sys ? sys[g_first[g]] : 0];
        double bl[3], bh[3], cc[3];
        float ch[3], cl[3], fl[3], fh[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            bl[a] = unord64(mlo[a]);
            bh[a] = unord64(mhi[a]);
            g_box[6 * g + a] = bl[a];
            g_box[6 * g + 3 + a] = bh[a];
            g_qbox[6 * g + a] = quantise(bl[a], bx.lo[a], bx.s);
            g_qbox[6 * g + 3 + a] = quantise(bh[a], bx.lo[a], bx.s);
            cc[a] = __dmul_rn(__dadd_rn(bl[a], bh[a]), 0.5);
            split_hilo(cc[a] - bx.c0[a], &ch[a], &cl[a]);
            fl[a] = __double2float_rd(bl[a] - cc[a]);
            fh[a] = __double2float_ru(bh[a] - cc[a]);
        }
        g_c64[g] = make_dvec4(cc[0], cc[1], cc[2], 0.0);
        g_ch[g] = make_float4(ch[0], ch[1], ch[2], 0.0f);
        g_cl[g] = make_float4(cl[0], cl[1], cl[2], 0.0f);
        g_blo[g] = make_float4(fl[0], fl[1], fl[2], 0.0f);
        g_bhi[g] = make_float4(fh[0], fh[1], fh[2], 0.0f);
    }
}

}  // namespace

int build_tree(fdps_tree* t, fdps_psys* ps) {
    fdps_ctx* ctx = t->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t n = ps->n;
    const int64_t ntiles = n > 0 ? (n + kBTile - 1) / kBTile : 1;
    const int64_t nw = ntiles * kBWarps;
    uint32_t* wcount = t->bt_count;                 // [21][nw] per warp
    uint32_t* tcount = wcount + kMaxLevel * nw;     // [21][ntiles] per tile, then scanned
    uint32_t* ltot = tcount + kMaxLevel * ntiles;   // [21]
    const RootArgs R{ps->n_sys, ps->d_off, n, t->p.n_leaf, t->nd_first, t->nd_count,
                     t->nd_child, t->nd_meta, t->nd_parent, t->nd_qlo};
    // per-position scratch: t->head, rewritten by the group selection
    k_tree_count<<<(unsigned)ntiles, kBT, 0, s>>>(n, t->p.n_leaf, t->keys_sorted, ps->d_sys, t->head, wcount,
                                                  tcount, nw, ntiles, R);
    FDPS_LAUNCH_CHECK(ctx);
    k_tree_scan<<<kMaxLevel, 1024, 0, s>>>(tcount, ntiles, ltot);
    FDPS_LAUNCH_CHECK(ctx);
    const unsigned grid_nodes = (unsigned)(n / kBTile + 1);  // positions 0 .. n
    k_tree_nodes<<<grid_nodes, kBT, 0, s>>>(n, ps->n_sys, t->cap_nodes, t->keys_sorted, ps->d_sys, t->head,
                                            wcount, tcount, nw, ntiles, ltot, t->st, t->nd_first, t->nd_count,
                                            t->nd_child, t->nd_meta, t->nd_parent, t->nd_qlo);
    FDPS_LAUNCH_CHECK(ctx);
    k_tree_finish<<<ctx->sm_count * 4, 256, 0, s>>>(t->st, ps->n_sys, t->nd_first, t->nd_count, t->nd_parent,
                                                    t->nd_child, t->nd_meta);
    FDPS_LAUNCH_CHECK(ctx);
    return FDPS_OK;
}

int compute_moments(fdps_tree* t, fdps_psys* ps) {
    fdps_ctx* ctx = t->ctx;
    const int c = ps->cur;
    MomArgs A;
    A.st = t->st;
    A.box = t->sys_box;
    A.sys = ps->d_sys;
    A.px = ps->x[c];
    A.py = ps->y[c];
    A.pz = ps->z[c];
    A.pm = ps->m[c];
    A.pmx = t->pmx;
    A.pmy = t->pmy;
    A.pmz = t->pmz;
    A.pf_hi = t->pf_hi;
    A.pf_lo = t->pf_lo;
    A.nd_first = t->nd_first;
    A.nd_count = t->nd_count;
    A.nd_child = t->nd_child;
    A.nd_meta = t->nd_meta;
    A.nd_parent = t->nd_parent;
    A.nd_qlo = t->nd_qlo;
    A.nd_sx = t->nd_sx;
    A.nd_sy = t->nd_sy;
    A.nd_sz = t->nd_sz;
    A.nd_com = t->nd_com;
    A.nd_quad = t->nd_quad;
    A.nd_f = t->nd_f;
    A.nd_walk = t->nd_walk;
    A.nd_fq0 = t->nd_fq0;
    A.nd_fq1 = t->nd_fq1;
    if (t->p.moment != FDPS_QUADRUPOLE) return launch_moments<false, false>(ctx, A, ps, t->st);
    if (t->p.precision == FDPS_FP64) return launch_moments<true, true>(ctx, A, ps, t->st);
    return launch_moments<true, false>(ctx, A, ps, t->st);
}

int select_groups(fdps_tree* t, fdps_psys* ps) {
    fdps_ctx* ctx = t->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t n = ps->n;
    const int c = ps->cur;
    const int G = t->box_blocks;
    FDPS_CUDA_TRY(ctx, cudaMemsetAsync(t->head, 0xFF, sizeof(uint32_t) * (size_t)n, s));
    k_group_mark<<<ctx->sm_count * 8, 256, 0, s>>>(t->st, t->p.n_grp, ps->n_sys, t->nd_first, t->nd_count,
                                                   t->nd_meta, t->nd_parent, t->head);
    FDPS_LAUNCH_CHECK(ctx);
    k_group_count<<<G, kB, 0, s>>>(n, t->head, t->grp_scan, t->st, t->cap_groups);
    FDPS_LAUNCH_CHECK(ctx);
    k_group_write<<<G, kB, 0, s>>>(n, t->cap_groups, t->head, t->grp_scan, t->nd_count, t->g_node,
                                   t->g_first, t->g_count);
    FDPS_LAUNCH_CHECK(ctx);
    k_group_data<<<ctx->sm_count * 8, 256, 0, s>>>(t->st, t->sys_box, ps->d_sys, t->g_first, t->g_count, ps->x[c],
                                                   ps->y[c], ps->z[c], t->g_box, t->g_qbox,
                                                   t->g_c64, t->g_ch, t->g_cl, t->g_blo, t->g_bhi);
    FDPS_LAUNCH_CHECK(ctx);
    return FDPS_OK;
}

}  // namespace fdps
