// keys_sort.cu -- root box, Morton keys, LSD radix sort and reorder.
//
// Tree construction of Sect. 3.2 starts from the particles' positions; the
// paper does not fix the key scheme.  This file implements the reading:
//   box   lo_a = min x_a, L = max_a (max x_a - lo_a) (1 if 0), s = 2^21 / L
//   key   q_a = min(2^21 - 1, floor((x_a - lo_a) * s)) with the subtraction
//         and the product each rounded to nearest in FP64 (no FMA), then
//         bits of q_x / q_y / q_z interleaved to key bits 3b+2 / 3b+1 / 3b
//   sort  stable by key: 8 LSD passes of 8-bit digits.  The force pipeline
//         takes the digit counts of all passes while it computes the keys,
//         then runs one kernel per pass (tile ranking, a bounded look-back
//         over earlier tiles for the global offsets, a staged scatter).
//         The allocation-free entry point keeps the reduce-then-scan form
//         (tile histograms, a scan, a stable scatter).
#include <atomic>

#include "fdps_internal.cuh"

namespace fdps {
namespace {

constexpr int kSortBlock = 256;
constexpr int kSortWarps = kSortBlock / 32;
constexpr int kSortKPT = 8;
constexpr int kSortTile = kSortBlock * kSortKPT;  // 2048 keys
constexpr int kRadix = 256;

// Order-preserving map of an FP64 value to an unsigned integer, so the
// box reduction runs on the integer pipes.  Min and max of the mapped
// values are the FP64 min and max (inputs are finite).
__device__ __forceinline__ unsigned long long ord64(double v) {
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double unord64(unsigned long long o) {
    unsigned long long u = (o >> 63) ? (o & 0x7FFFFFFFFFFFFFFFull) : ~o;
    return __longlong_as_double((long long)u);
}

constexpr int kBoxBlock = 512;  // threads per block of the root-box reduction

__global__ void __launch_bounds__(kBoxBlock, 4) k_box_partial(int64_t n, const double* __restrict__ x,
                                                     const double* __restrict__ y,
                                                     const double* __restrict__ z,
                                                     BoxPartial* __restrict__ part) {
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull};
    unsigned long long hi[3] = {0ull, 0ull, 0ull};
    auto take = [&](double vx, double vy, double vz) {
        const unsigned long long o[3] = {ord64(vx), ord64(vy), ord64(vz)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = o[a] < lo[a] ? o[a] : lo[a];
            hi[a] = o[a] > hi[a] ? o[a] : hi[a];
        }
    };
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if ((((uintptr_t)x | (uintptr_t)y | (uintptr_t)z) & 15) == 0) {
        // 16-byte loads, two pairs of particles in flight per thread
        const double2* x2 = reinterpret_cast<const double2*>(x);
        const double2* y2 = reinterpret_cast<const double2*>(y);
        const double2* z2 = reinterpret_cast<const double2*>(z);
        const int64_t n2 = n >> 1;
        int64_t p = t0;
        for (; p + G < n2; p += 2 * G) {
            const double2 a0 = x2[p], b0 = y2[p], c0 = z2[p];
            const double2 a1 = x2[p + G], b1 = y2[p + G], c1 = z2[p + G];
            take(a0.x, b0.x, c0.x);
            take(a0.y, b0.y, c0.y);
            take(a1.x, b1.x, c1.x);
            take(a1.y, b1.y, c1.y);
        }
        for (; p < n2; p += G) {
            const double2 a0 = x2[p], b0 = y2[p], c0 = z2[p];
            take(a0.x, b0.x, c0.x);
            take(a0.y, b0.y, c0.y);
        }
        if ((n & 1) && t0 == 0) take(x[n - 1], y[n - 1], z[n - 1]);
    } else {
        for (int64_t i = t0; i < n; i += G) take(x[i], y[i], z[i]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            unsigned long long l = __shfl_xor_sync(0xFFFFFFFFu, lo[a], off);
            unsigned long long h = __shfl_xor_sync(0xFFFFFFFFu, hi[a], off);
            lo[a] = l < lo[a] ? l : lo[a];
            hi[a] = h > hi[a] ? h : hi[a];
        }
    }
    __shared__ unsigned long long s_lo[kBoxBlock / 32][3], s_hi[kBoxBlock / 32][3];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) {
            s_lo[w][a] = lo[a];
            s_hi[w][a] = hi[a];
        }
    __syncthreads();
    if (threadIdx.x < 3) {
        int a = threadIdx.x;
        unsigned long long l = s_lo[0][a], h = s_hi[0][a];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            l = s_lo[k][a] < l ? s_lo[k][a] : l;
            h = s_hi[k][a] > h ? s_hi[k][a] : h;
        }
        // blocks that saw no particle keep the neutral sentinels
        part[blockIdx.x].lo[a] = __longlong_as_double((long long)l);
        part[blockIdx.x].hi[a] = __longlong_as_double((long long)h);
    }
}

// One warp: lanes reduce strided subsets of the block partials, then the
// lanes' results are combined by shuffles.
__global__ void k_box_final(int nparts, const BoxPartial* __restrict__ part, DevState* st,
                            SysBox* box) {
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    for (int b = threadIdx.x; b < nparts; b += 32)
        for (int a = 0; a < 3; ++a) {
            unsigned long long l = (unsigned long long)__double_as_longlong(part[b].lo[a]);
            unsigned long long h = (unsigned long long)__double_as_longlong(part[b].hi[a]);
            lo[a] = l < lo[a] ? l : lo[a];
            hi[a] = h > hi[a] ? h : hi[a];
        }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const unsigned long long l = __shfl_xor_sync(0xFFFFFFFFu, lo[a], off);
            const unsigned long long h = __shfl_xor_sync(0xFFFFFFFFu, hi[a], off);
            lo[a] = l < lo[a] ? l : lo[a];
            hi[a] = h > hi[a] ? h : hi[a];
        }
    if (threadIdx.x != 0) return;
    double L = 0.0;
    for (int a = 0; a < 3; ++a) {
        double l = unord64(lo[a]), h = unord64(hi[a]);
        st->lo[a] = l;
        double e = __dsub_rn(h, l);
        L = e > L ? e : L;
    }
    if (L == 0.0) L = 1.0;
    st->L = L;
    st->s = __ddiv_rn(2097152.0, L);
    for (int a = 0; a < 3; ++a) st->c0[a] = __dadd_rn(st->lo[a], __dmul_rn(0.5, L));
    for (int a = 0; a < 3; ++a) {
        box->lo[a] = st->lo[a];
        box->c0[a] = st->c0[a];
    }
    box->L = st->L;
    box->s = st->s;
}

// Root boxes of independent systems: one block per system (positions
// off[k] .. off[k+1]), the same definitions as for a single system.
__global__ void __launch_bounds__(256) k_box_seg(const int64_t* __restrict__ off,
                                                 const double* __restrict__ x,
                                                 const double* __restrict__ y,
                                                 const double* __restrict__ z,
                                                 SysBox* __restrict__ box) {
    const int64_t a0 = off[blockIdx.x], a1 = off[blockIdx.x + 1];
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull};
    unsigned long long hi[3] = {0ull, 0ull, 0ull};
    for (int64_t i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
        unsigned long long v[3] = {ord64(x[i]), ord64(y[i]), ord64(z[i])};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = v[a] < lo[a] ? v[a] : lo[a];
            hi[a] = v[a] > hi[a] ? v[a] : hi[a];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            unsigned long long l = __shfl_xor_sync(0xFFFFFFFFu, lo[a], o);
            unsigned long long h = __shfl_xor_sync(0xFFFFFFFFu, hi[a], o);
            lo[a] = l < lo[a] ? l : lo[a];
            hi[a] = h > hi[a] ? h : hi[a];
        }
    __shared__ unsigned long long s_lo[8][3], s_hi[8][3];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) {
            s_lo[w][a] = lo[a];
            s_hi[w][a] = hi[a];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        double L = 0.0, l3[3];
        for (int a = 0; a < 3; ++a) {
            unsigned long long l = s_lo[0][a], h = s_hi[0][a];
            for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
                l = s_lo[k][a] < l ? s_lo[k][a] : l;
                h = s_hi[k][a] > h ? s_hi[k][a] : h;
            }
            l3[a] = unord64(l);
            const double e = __dsub_rn(unord64(h), l3[a]);
            L = e > L ? e : L;
        }
        if (L == 0.0) L = 1.0;
        SysBox b;
        for (int a = 0; a < 3; ++a) b.lo[a] = l3[a];
        b.L = L;
        b.s = __ddiv_rn(2097152.0, L);
        for (int a = 0; a < 3; ++a) b.c0[a] = __dadd_rn(l3[a], __dmul_rn(0.5, L));
        box[blockIdx.x] = b;
    }
}


// Spread the low 21 bits of v to every third bit (bit b -> bit 3b).
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1FFFFFu;
    x = (x | (x << 32)) & 0x001F00000000FFFFull;
    x = (x | (x << 16)) & 0x001F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Keys of one 2048-key tile per block, plus that tile's histogram of the
// lowest digit (the first sort pass).
__global__ void __launch_bounds__(kSortBlock) k_keys(int64_t n, const double* __restrict__ x,
                                                     const double* __restrict__ y,
                                                     const double* __restrict__ z,
                                                     const SysBox* __restrict__ box,
                                                     const uint32_t* __restrict__ sys,
                                                     uint64_t* __restrict__ keys,
                                                     uint32_t* __restrict__ hist, int ntiles) {
    __shared__ uint32_t h[kSortWarps][kRadix];
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortBlock) (&h[0][0])[i] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = (int64_t)blockIdx.x * kSortTile + w * (32 * kSortKPT);
#pragma unroll
    for (int r = 0; r < kSortKPT; ++r) {
        int64_t i = base + r * 32 + lane;
        if (i < n) {
            const SysBox& b = box[sys ? sys[i] : 0];
            uint32_t qx = quantise(x[i], b.lo[0], b.s), qy = quantise(y[i], b.lo[1], b.s),
                     qz = quantise(z[i], b.lo[2], b.s);
            uint64_t k = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
            keys[i] = k;
            atomicAdd(&h[w][k & 0xFF], 1u);
        }
    }
    __syncthreads();
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kSortWarps; ++k) c += h[k][threadIdx.x];
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = c;
}

__global__ void __launch_bounds__(kSortBlock) k_radix_hist(int64_t n, const uint64_t* __restrict__ keys,
                                                           int shift, uint32_t* __restrict__ hist,
                                                           int ntiles) {
    __shared__ uint32_t h[kSortWarps][kRadix];
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortBlock) (&h[0][0])[i] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = (int64_t)blockIdx.x * kSortTile + w * (32 * kSortKPT);
#pragma unroll
    for (int r = 0; r < kSortKPT; ++r) {
        int64_t i = base + r * 32 + lane;
        if (i < n) atomicAdd(&h[w][(keys[i] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kSortWarps; ++k) c += h[k][threadIdx.x];
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = c;
}

// Exclusive block scan of one value per thread (blockDim.x <= 1024); the
// block total is kept apart from the 32 per-warp offsets.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
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
    if (total) *total = s_w[32];
    __syncthreads();
    return res;
}

// One block per digit: exclusive scan of that digit's row of tile counts.
__global__ void __launch_bounds__(1024) k_radix_scan_rows(uint32_t* __restrict__ hist, int ntiles,
                                                          uint32_t* __restrict__ dtot) {
    uint32_t* row = hist + (int64_t)blockIdx.x * ntiles;
    const int per = (ntiles + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per;
    uint32_t sum = 0;
    for (int k = 0; k < per; ++k)
        if (b + k < ntiles) sum += row[b + k];
    uint32_t total;
    uint32_t off = block_excl_scan(sum, &total);
    for (int k = 0; k < per; ++k)
        if (b + k < ntiles) {
            uint32_t c = row[b + k];
            row[b + k] = off;
            off += c;
        }
    if (threadIdx.x == 0) dtot[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kRadix) k_radix_scan_digits(uint32_t* __restrict__ dtot) {
    uint32_t v = dtot[threadIdx.x];
    uint32_t off = block_excl_scan(v, nullptr);
    dtot[threadIdx.x] = off;
}

// Stable scatter of one tile: warp-level ranking with match_any, tile-local
// reordering in shared memory, then coalesced runs per digit.
__global__ void __launch_bounds__(kSortBlock) k_radix_scatter(
    int64_t n, const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
    uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int shift,
    const uint32_t* __restrict__ hist, const uint32_t* __restrict__ dbase, int ntiles,
    const uint32_t* __restrict__ sys = nullptr) {
    __shared__ uint64_t sk[kSortTile];
    __shared__ uint32_t sv[kSortTile];
    __shared__ uint8_t sd[kSortTile];
    __shared__ uint32_t wcnt[kSortWarps][kRadix];
    __shared__ uint32_t tstart[kRadix];
    __shared__ uint32_t gbase[kRadix];
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortBlock) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    const int64_t base = tile0 + w * (32 * kSortKPT);
    uint64_t mk[kSortKPT];
    uint32_t mv[kSortKPT], mr[kSortKPT], md[kSortKPT];
#pragma unroll
    for (int r = 0; r < kSortKPT; ++r) {
        int64_t i = base + r * 32 + lane;
        bool valid = i < n;
        uint64_t k = valid ? kin[i] : 0ull;
        uint32_t v = valid ? (vin ? vin[i] : (uint32_t)i) : 0u;
        uint32_t d = sys ? (valid ? (sys[v] >> shift) & 0xFFu : 0u) : (uint32_t)(k >> shift) & 0xFFu;
        uint32_t vmask = __ballot_sync(0xFFFFFFFFu, valid);
        uint32_t rank = 0, before = 0, peers = 0;
        if (valid) {
            peers = __match_any_sync(vmask, d);
            rank = __popc(peers & lt_mask);
            before = wcnt[w][d];
        }
        __syncwarp();
        if (valid && rank == 0) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
        mk[r] = k;
        mv[r] = v;
        mr[r] = before + rank;
        md[r] = d;
    }
    __syncthreads();
    {
        const int d = threadIdx.x;  // one thread per digit
        uint32_t run = 0;
#pragma unroll
        for (int k = 0; k < kSortWarps; ++k) {
            uint32_t c = wcnt[k][d];
            wcnt[k][d] = run;
            run += c;
        }
        uint32_t st0 = block_excl_scan(run, nullptr);
        tstart[d] = st0;
        gbase[d] = dbase[d] + hist[(int64_t)d * ntiles + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortKPT; ++r) {
        int64_t i = base + r * 32 + lane;
        if (i < n) {
            const uint32_t d = md[r];
            uint32_t p = tstart[d] + wcnt[w][d] + mr[r];
            sk[p] = mk[r];
            sv[p] = mv[r];
            sd[p] = (uint8_t)md[r];
        }
    }
    __syncthreads();
    int64_t rem = n - tile0;
    const int cnt = rem < kSortTile ? (int)rem : kSortTile;
    for (int p = threadIdx.x; p < cnt; p += kSortBlock) {
        uint64_t k = sk[p];
        const uint32_t d = sd[p];
        uint32_t dst = gbase[d] + (uint32_t)p - tstart[d];
        kout[dst] = k;
        vout[dst] = sv[p];
    }
}

// ---------------------------------------------- single-pass radix passes
//
// The force pipeline sorts with one kernel per digit pass: the digit
// histograms of every pass are taken up front (they do not depend on the
// order), and within a pass each 2048-key tile learns where its keys go by
// looking back over the tiles before it ("decoupled look-back": every tile
// publishes its per-digit count, then its inclusive prefix once known).
// Tiles take their index in the order they start, so a tile only ever
// waits on tiles already running; every wait is bounded and gives up with
// an error flag instead of spinning on.

constexpr uint32_t kFlagAgg = 1u << 30;   // tile count published
constexpr uint32_t kFlagInc = 1u << 31;   // inclusive prefix published
constexpr uint32_t kValMask = kFlagAgg - 1u;
constexpr int kMaxSpin = 1 << 20;
constexpr int kHistBlocks = 608;

// Morton keys (as k_keys) plus the histograms of all digit passes: hist
// [pass][256] with passes 0..7 the key bytes and, for several systems,
// passes 8, 9 the two low bytes of the system id.  The last block to finish
// (counted in *done, zero on entry) turns every pass's counts into the
// exclusive digit bases.
__global__ void __launch_bounds__(kSortBlock) k_keys_hist(int64_t n, const double* __restrict__ x,
                                                          const double* __restrict__ y,
                                                          const double* __restrict__ z,
                                                          const SysBox* __restrict__ box,
                                                          const uint32_t* __restrict__ sys,
                                                          uint64_t* __restrict__ keys,
                                                          uint32_t* __restrict__ hist, uint32_t* done) {
    __shared__ bool s_last;
    __shared__ uint32_t h[10][kRadix];
    for (int i = threadIdx.x; i < 10 * kRadix; i += kSortBlock) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t sid = sys ? sys[i] : 0u;
        const SysBox& b = box[sid];
        const uint32_t qx = quantise(x[i], b.lo[0], b.s), qy = quantise(y[i], b.lo[1], b.s),
                       qz = quantise(z[i], b.lo[2], b.s);
        const uint64_t k = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
        keys[i] = k;
#pragma unroll
        for (int p = 0; p < 8; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 0xFF], 1u);
        if (sys) {
            atomicAdd(&h[8][sid & 0xFF], 1u);
            atomicAdd(&h[9][(sid >> 8) & 0xFF], 1u);
        }
    }
    __syncthreads();
    const int np = sys ? 10 : 8;
    for (int i = threadIdx.x; i < np * kRadix; i += kSortBlock) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
    __threadfence();  // this block's counts are in hist before it counts itself done
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last block: exclusive scan of each pass's 256 digit counts
    static_assert(kSortBlock == kRadix, "one thread per digit");
    for (int p = 0; p < np; ++p) {
        uint32_t* row = hist + p * kRadix;
        const uint32_t v = __ldcg(&row[threadIdx.x]);
        row[threadIdx.x] = block_excl_scan(v, nullptr);
    }
}

// ------------------------------------------------ coherent time-step sort
//
// In time stepping the particles enter each sort in the previous call's key
// order and move little in one step.  The previous call's sorted keys at
// every kCohT-th position are then splitters that put almost every particle
// in the bucket of its own position: bucket b holds the keys in
// [prev[b kCohT], prev[(b + 1) kCohT]) (bucket 0 from 0, the last bucket
// to the end).  Three passes give the stable permutation of the radix sort:
// keys, buckets and bucket counts (the last block scans the counts into
// offsets and checks that every bucket fits one CTA), a scatter into the
// buckets, and a merge sort of each bucket in shared memory by (key,
// position).  A bucket above kCohCap keys
// sets kSortRedo: the kernels after the sort treat the call's order as
// unsorted and the host redoes the call with the radix sort.

constexpr int kCohCap = 2048; // largest bucket one CTA sorts
constexpr int kCohBlock = 256;
constexpr int kCohWarps = kCohBlock / 32;
constexpr int kCohNear = 2;   // buckets t - 2 .. t + 2 counted in shared memory
static_assert(kCohT % kCohBlock == 0, "whole rounds per tile");

// Where the buckets lie: bucket b takes the positions [start(b), start(b +
// 1)) of the previous order, of system sys(b); the buckets of system k are
// first(k) .. first(k + 1) - 1 and never cross a system's segment (the
// systems keep their segments from call to call).  One system: start(b) =
// b kCohT (the last bucket ragged), no tables.
struct CohLayout {
    const uint32_t* start;  // [nb + 1], or null
    const uint32_t* sys;    // [nb], or null (system 0)
    const uint32_t* first;  // [n_sys + 1], or null ({0, nb})
    uint32_t nb;
    int64_t n;
};
__device__ __forceinline__ int64_t coh_start(const CohLayout& L, uint32_t b) {
    if (L.start) return (int64_t)L.start[b];
    const int64_t p = (int64_t)b * kCohT;
    return p < L.n ? p : L.n;
}

// The splitter of bucket j (above its system's first bucket) is
// prev[start(j)]; the bucket of key k in system buckets [j0, j1) is the
// largest j with splitter(j) <= k (splitter(j0) = 0), starting from t.
__device__ __forceinline__ uint32_t coh_bucket(uint64_t k, uint32_t t, uint32_t j0, uint32_t j1,
                                               const uint64_t* __restrict__ prev, const CohLayout& L) {
    const uint64_t lo = t == j0 ? 0ull : prev[coh_start(L, t)];
    const bool below_hi = t + 1 >= j1 || k < prev[coh_start(L, t + 1)];
    if (k >= lo && below_hi) return t;
    uint32_t a, z;  // the answer lies in [a, z); splitter(a) <= k
    if (k < lo) {
        a = j0;
        z = t;
    } else {
        a = t + 1;
        z = j1;
    }
    while (z - a > 1) {
        const uint32_t mid = (a + z) >> 1;
        if (prev[coh_start(L, mid)] <= k)
            a = mid;
        else
            z = mid;
    }
    return a;
}

// Pass 1 (one block per bucket's positions, at most kCohT): Morton keys as
// k_keys, the bucket of every key, bucket counts; the last block turns the
// counts into offsets and cursors and flags a bucket above kCohCap.
__global__ void __launch_bounds__(kCohBlock) k_coh_keys(CohLayout L, const double* __restrict__ x,
                                                        const double* __restrict__ y,
                                                        const double* __restrict__ z,
                                                        const SysBox* __restrict__ box,
                                                        const uint64_t* __restrict__ prev,
                                                        uint64_t* __restrict__ keys, uint32_t* __restrict__ bkt,
                                                        uint32_t* cnt, uint32_t* off, uint32_t* cur,
                                                        uint32_t* done, uint32_t* err) {
    __shared__ uint32_t s_near[2 * kCohNear + 1];
    __shared__ uint32_t s_max[kCohWarps];
    __shared__ bool s_last;
    const uint32_t t = blockIdx.x;
    const uint32_t nb = L.nb;
    if (threadIdx.x < 2 * kCohNear + 1) s_near[threadIdx.x] = 0;
    __syncthreads();
    const int64_t p0 = coh_start(L, t), p1 = coh_start(L, t + 1);
    const uint32_t sys = L.sys ? L.sys[t] : 0u;
    const uint32_t j0 = L.first ? L.first[sys] : 0u, j1 = L.first ? L.first[sys + 1] : nb;
    const SysBox& b = box[sys];
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < kCohT / kCohBlock; ++r) {
        const int64_t i = p0 + r * kCohBlock + threadIdx.x;
        int d = 0x7FFFFFFF;  // no particle
        if (i < p1) {
            const uint32_t qx = quantise(x[i], b.lo[0], b.s), qy = quantise(y[i], b.lo[1], b.s),
                           qz = quantise(z[i], b.lo[2], b.s);
            const uint64_t k = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
            keys[i] = k;
            const uint32_t bk = coh_bucket(k, t, j0, j1, prev, L);
            bkt[i] = bk;
            d = (int)bk - (int)t;
            if (d < -kCohNear || d > kCohNear) atomicAdd(&cnt[bk], 1u);
        }
        // one shared atomic per warp and nearby bucket
#pragma unroll
        for (int v = -kCohNear; v <= kCohNear; ++v) {
            const uint32_t mk = __ballot_sync(0xFFFFFFFFu, d == v);
            if (mk && lane == __ffs(mk) - 1) atomicAdd(&s_near[v + kCohNear], (uint32_t)__popc(mk));
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * kCohNear + 1) {
        const int bk = (int)t + (int)threadIdx.x - kCohNear;
        const uint32_t c = s_near[threadIdx.x];
        if (c && bk >= 0 && bk < (int)nb) atomicAdd(&cnt[bk], c);
    }
    __threadfence();  // this block's counts land before it counts itself done
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // exclusive scan of the counts in rounds of 4 kCohBlock consecutive
    // buckets (4 per thread), the next round's counts loaded ahead
    constexpr int kRound = 4 * kCohBlock;
    uint32_t carry = 0, mx = 0, c[4], cn[4];
    auto load4 = [&](int r0, uint32_t* v) {
        const int j = r0 + 4 * (int)threadIdx.x;
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = j + q < (int)nb ? __ldcg(&cnt[j + q]) : 0u;
    };
    load4(0, c);
    for (int r0 = 0; r0 < (int)nb; r0 += kRound) {
        load4(r0 + kRound, cn);
        uint32_t tot;
        uint32_t o = carry + block_excl_scan(c[0] + c[1] + c[2] + c[3], &tot);
        const int j = r0 + 4 * (int)threadIdx.x;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (j + q < (int)nb) {
                off[j + q] = o;
                cur[j + q] = o;
            }
            o += c[q];
            mx = c[q] > mx ? c[q] : mx;
            c[q] = cn[q];
        }
        carry += tot;
    }
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        off[nb] = carry;
        uint32_t m = 0;
        for (int w = 0; w < kCohWarps; ++w) m = s_max[w] > m ? s_max[w] : m;
        if (m > (uint32_t)kCohCap) atomicOr(err, kSortRedo);
    }
}

// Pass 2: every (key, position) into its bucket; one atomic per block and
// nearby bucket reserves the block's slots, far movers take one each.  The
// order inside a bucket is arbitrary (pass 3 sorts by position too).
__global__ void __launch_bounds__(kCohBlock) k_coh_scatter(CohLayout L, const uint64_t* __restrict__ keys,
                                                           const uint32_t* __restrict__ bkt,
                                                           uint32_t* cur, uint64_t* __restrict__ k2,
                                                           uint32_t* __restrict__ i2, const uint32_t* err) {
    constexpr int R = kCohT / kCohBlock;
    __shared__ uint32_t s_cnt[2 * kCohNear + 1], s_base[2 * kCohNear + 1];
    if (*err & kSortRedo) return;
    const uint32_t t = blockIdx.x;
    const uint32_t nb = L.nb;
    const int64_t p0 = coh_start(L, t), p1 = coh_start(L, t + 1);
    if (threadIdx.x < 2 * kCohNear + 1) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    uint64_t kk[R];
    uint32_t bb[R], rank[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = p0 + r * kCohBlock + threadIdx.x;
        bb[r] = 0xFFFFFFFFu;
        rank[r] = 0xFFFFFFFFu;
        kk[r] = 0;
        if (i < p1) {
            kk[r] = keys[i];
            bb[r] = bkt[i];
        }
        // ranks among this block's pairs for the nearby buckets: one shared
        // atomic per warp and bucket, lanes ranked by the ballot
        const int d = bb[r] == 0xFFFFFFFFu ? 0x7FFFFFFF : (int)bb[r] - (int)t;
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int v = -kCohNear; v <= kCohNear; ++v) {
            const uint32_t mk = __ballot_sync(0xFFFFFFFFu, d == v);
            if (mk) {
                const int lead = __ffs(mk) - 1;
                uint32_t base = 0;
                if (lane == lead) base = atomicAdd(&s_cnt[v + kCohNear], (uint32_t)__popc(mk));
                base = __shfl_sync(0xFFFFFFFFu, base, lead);
                if (d == v) rank[r] = base + (uint32_t)__popc(mk & ((1u << lane) - 1u));
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * kCohNear + 1) {
        const int bk = (int)t + (int)threadIdx.x - kCohNear;
        const uint32_t c = s_cnt[threadIdx.x];
        s_base[threadIdx.x] = (c && bk >= 0 && bk < (int)nb) ? atomicAdd(&cur[bk], c) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (bb[r] == 0xFFFFFFFFu) continue;
        const int64_t i = p0 + r * kCohBlock + threadIdx.x;
        const uint32_t pos = rank[r] != 0xFFFFFFFFu ? s_base[(int)bb[r] - (int)t + kCohNear] + rank[r]
                                                    : atomicAdd(&cur[bb[r]], 1u);
        k2[pos] = kk[r];
        i2[pos] = (uint32_t)i;
    }
}

// Shared memory of the bucket sort: two key and two position buffers,
// element j at j + j / 16 (keys) and j + j / 32 (positions), so that the
// threads of a warp reading or writing their EPT consecutive elements fall
// in different banks.
constexpr int kCohKP = kCohCap + kCohCap / 16;
constexpr int kCohIP = kCohCap + kCohCap / 32;
struct CohShared {
    unsigned long long k[2][kCohKP];
    uint32_t i[2][kCohIP];
};
__device__ __forceinline__ int coh_kp(int j) { return j + (j >> 4); }
__device__ __forceinline__ int coh_ip(int j) { return j + (j >> 5); }

// (key, position) order: all pairs of a call differ, so any correct sort of
// them is the stable sort by key.  The padding pair (all ones) orders last.
__device__ __forceinline__ bool coh_less(unsigned long long ka, uint32_t ia, unsigned long long kb, uint32_t ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// Merge sort of kCohBlock * EPT pairs in buffer 0: each thread sorts its
// EPT consecutive pairs in registers, then every round merges runs of
// length L pairwise (L = EPT, 2 EPT, ...), each thread writing EPT
// consecutive outputs from the split of its output diagonal found by
// binary search (merge path).  Returns the buffer holding the result.
template <int EPT>
__device__ __noinline__ int coh_merge_sort(CohShared& sm) {
    constexpr int np = kCohBlock * EPT;
    const int o = threadIdx.x * EPT;
    {
        unsigned long long k[EPT];
        uint32_t x[EPT];
#pragma unroll
        for (int r = 0; r < EPT; ++r) {
            k[r] = sm.k[0][coh_kp(o + r)];
            x[r] = sm.i[0][coh_ip(o + r)];
        }
        // odd-even transposition sort
#pragma unroll
        for (int p = 0; p < EPT; ++p)
#pragma unroll
            for (int r = p & 1; r + 1 < EPT; r += 2)
                if (coh_less(k[r + 1], x[r + 1], k[r], x[r])) {
                    const unsigned long long tk = k[r];
                    k[r] = k[r + 1];
                    k[r + 1] = tk;
                    const uint32_t tx = x[r];
                    x[r] = x[r + 1];
                    x[r + 1] = tx;
                }
#pragma unroll
        for (int r = 0; r < EPT; ++r) {
            sm.k[0][coh_kp(o + r)] = k[r];
            sm.i[0][coh_ip(o + r)] = x[r];
        }
    }
    __syncthreads();
    int src = 0;
    for (int L = EPT; L < np; L *= 2) {
        const int a0 = (o / (2 * L)) * (2 * L);  // run A is [a0, a0 + L), run B follows
        const int b0 = a0 + L;
        const int d = o - a0;
        const unsigned long long* K = sm.k[src];
        const uint32_t* X = sm.i[src];
        // ia = how many of the first d outputs come from A
        int lo = d > L ? d - L : 0, hi = d < L ? d : L;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            const int jb = b0 + d - 1 - mid;
            if (coh_less(K[coh_kp(a0 + mid)], X[coh_ip(a0 + mid)], K[coh_kp(jb)], X[coh_ip(jb)]))
                lo = mid + 1;
            else
                hi = mid;
        }
        int ia = lo, ib = d - lo;
        unsigned long long ka = K[coh_kp(a0 + min(ia, L - 1))], kb = K[coh_kp(b0 + min(ib, L - 1))];
        uint32_t xa = X[coh_ip(a0 + min(ia, L - 1))], xb = X[coh_ip(b0 + min(ib, L - 1))];
        unsigned long long* OK = sm.k[src ^ 1];
        uint32_t* OX = sm.i[src ^ 1];
#pragma unroll
        for (int r = 0; r < EPT; ++r) {
            const bool ta = ib >= L || (ia < L && coh_less(ka, xa, kb, xb));
            OK[coh_kp(o + r)] = ta ? ka : kb;
            OX[coh_ip(o + r)] = ta ? xa : xb;
            if (ta) {
                ++ia;
                const int j = a0 + min(ia, L - 1);
                ka = K[coh_kp(j)];
                xa = X[coh_ip(j)];
            } else {
                ++ib;
                const int j = b0 + min(ib, L - 1);
                kb = K[coh_kp(j)];
                xb = X[coh_ip(j)];
            }
        }
        __syncthreads();
        src ^= 1;
    }
    return src;
}

// Pass 3 (one block per bucket): the bucket's m pairs, padded to
// kCohBlock * EPT with EPT = ceil(m / kCohBlock), sorted by (key, position)
// in shared memory and written to their final slots.
__global__ void __launch_bounds__(kCohBlock) k_coh_sort(const uint32_t* __restrict__ off, uint32_t nb,
                                                        const uint64_t* __restrict__ k2,
                                                        const uint32_t* __restrict__ i2,
                                                        uint64_t* __restrict__ keys_out,
                                                        uint32_t* __restrict__ perm_out, const uint32_t* err) {
    extern __shared__ __align__(16) unsigned char coh_dsm[];
    CohShared& sm = *reinterpret_cast<CohShared*>(coh_dsm);
    if (*err & kSortRedo) return;
    const uint32_t b = blockIdx.x;
    const uint32_t a0 = off[b];
    const int m = (int)(off[b + 1] - a0);
    if (m > kCohCap || m == 0) return;  // an overflow is flagged by pass 1
    const int ept = (m + kCohBlock - 1) / kCohBlock;
    const int np = ept * kCohBlock;
    for (int j = threadIdx.x; j < np; j += kCohBlock) {
        const bool v = j < m;
        sm.k[0][coh_kp(j)] = v ? k2[a0 + j] : ~0ull;
        sm.i[0][coh_ip(j)] = v ? i2[a0 + j] : 0xFFFFFFFFu;
    }
    __syncthreads();
    static_assert(kCohCap == 8 * kCohBlock, "at most 8 pairs a thread");
    int src = 0;
    switch (ept) {
        case 1: src = coh_merge_sort<1>(sm); break;
        case 2: src = coh_merge_sort<2>(sm); break;
        case 3: src = coh_merge_sort<3>(sm); break;
        case 4: src = coh_merge_sort<4>(sm); break;
        case 5: src = coh_merge_sort<5>(sm); break;
        case 6: src = coh_merge_sort<6>(sm); break;
        case 7: src = coh_merge_sort<7>(sm); break;
        default: src = coh_merge_sort<8>(sm); break;
    }
    for (int j = threadIdx.x; j < m; j += kCohBlock) {
        keys_out[a0 + j] = sm.k[src][coh_kp(j)];
        perm_out[a0 + j] = sm.i[src][coh_ip(j)];
    }
}

// Tile shape of the single-pass kernel and the look-back window: each
// look-back step reads the statuses of kLook earlier tiles at once.
constexpr int kOsBlock = 256;
constexpr int kOsKPT = 12;
constexpr int kOsTile = kOsBlock * kOsKPT;
constexpr int kOsMinBlocks = 3;
constexpr int kLook = 8;
// the look-back status buffer is sized for tiles of at least 2048 keys
static_assert(kOsTile >= 2048, "status rows sized for 2048-key tiles");

constexpr uint32_t kFlags = kFlagInc | kFlagAgg;
// Warp ranking by one match instruction per key (else eight ballots).
constexpr bool kRankMatch = false;

// One tile of one pass.  FULL tiles hold kOsTile keys and skip every bound
// check; the last tile of a pass may be ragged.  Indices fit in 32 bits
// (the tree takes fewer than 2^30 particles).
template <bool SYSKEY, bool FULL>
__device__ __forceinline__ void onesweep_tile(
    const int n, const int tile, const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
    uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, const int shift,
    const uint32_t* __restrict__ dbase, volatile uint32_t* st, uint32_t* __restrict__ st_next,
    const uint32_t* __restrict__ sys, uint32_t* err, uint64_t* sk, uint32_t* sv, uint8_t* sd,
    uint32_t (*wcnt)[kRadix], uint32_t* tstart, uint32_t* gdelta) {
    constexpr int kWarps = kOsBlock / 32;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int tile0 = tile * kOsTile;
    const int nv = FULL ? kOsTile : min(n - tile0, kOsTile);  // keys in this tile
    const int wb = w * (32 * kOsKPT);                         // the warp's first key
    // all loads of the tile first, so they are in flight together
    uint64_t mk[kOsKPT];
    uint32_t mv[kOsKPT], mr[kOsKPT];
#pragma unroll
    for (int r = 0; r < kOsKPT; ++r) {
        const int o = wb + r * 32 + lane;
        const bool ok = FULL || o < nv;
        mk[r] = ok ? kin[tile0 + o] : 0ull;
        mv[r] = ok ? (vin ? vin[tile0 + o] : (uint32_t)(tile0 + o)) : 0u;
    }
    uint32_t md[SYSKEY ? kOsKPT : 1];
    if (SYSKEY) {
#pragma unroll
        for (int r = 0; r < kOsKPT; ++r)
            md[r] = (FULL || wb + r * 32 + lane < nv) ? (sys[mv[r]] >> shift) & 0xFFu : 0u;
    }
    auto digit = [&](int r) -> uint32_t {
        return SYSKEY ? md[r] : (uint32_t)(mk[r] >> shift) & 0xFFu;
    };
    // lanes holding the same digit; invalid lanes get an empty mask
#pragma unroll
    for (int r = 0; r < kOsKPT; ++r) {
        const bool ok = FULL || wb + r * 32 + lane < nv;
        const uint32_t d = digit(r);
        uint32_t peers;
        if (kRankMatch) {
            peers = __match_any_sync(0xFFFFFFFFu, ok ? d : 0x100u);
        } else {
            peers = FULL ? 0xFFFFFFFFu : __ballot_sync(0xFFFFFFFFu, ok);
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const uint32_t bb = __ballot_sync(0xFFFFFFFFu, (d >> b) & 1u);
                peers &= ((d >> b) & 1u) ? bb : ~bb;
            }
        }
        mr[r] = ok ? peers : 0u;
    }
    // running per-warp digit counts, in key order: the first lane of each
    // digit group reads and advances the counter, the group takes its base
#pragma unroll
    for (int r = 0; r < kOsKPT; ++r) {
        const uint32_t peers = mr[r], d = digit(r);
        const uint32_t rank = __popc(peers & lt_mask);
        uint32_t b0 = 0;
        if (peers && rank == 0) {
            b0 = wcnt[w][d];
            wcnt[w][d] = b0 + __popc(peers);
        }
        __syncwarp();
        b0 = __shfl_sync(0xFFFFFFFFu, b0, (__ffs(peers) - 1) & 31);
        mr[r] = b0 + rank;
    }
    __syncthreads();
    // threads below kRadix own one digit each from here to the scatter
    const int d = threadIdx.x;
    uint32_t run = 0;
    if (d < kRadix) {
#pragma unroll
        for (int k = 0; k < kWarps; ++k) {
            const uint32_t c = wcnt[k][d];
            wcnt[k][d] = run;
            run += c;
        }
        // publish this tile's count at once, so later tiles can look past it
        st[(size_t)tile * kRadix + d] = (tile == 0 ? kFlagInc : kFlagAgg) | run;
        // the next pass looks back in the other buffer: clear this tile's row
        st_next[(size_t)tile * kRadix + d] = 0u;
    }
    const uint32_t ts = block_excl_scan(run, nullptr);
    if (d < kRadix) tstart[d] = ts;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kOsKPT; ++r) {
        if (FULL || wb + r * 32 + lane < nv) {
            const uint32_t dd = digit(r);
            const uint32_t p = tstart[dd] + wcnt[w][dd] + mr[r];
            sk[p] = mk[r];
            sv[p] = mv[r];
            if (SYSKEY) sd[p] = (uint8_t)dd;
        }
    }
    // look back over the tiles before this one for the keys of digit d:
    // add published counts, newest first, until an inclusive prefix.  A
    // window of kLook statuses is read at once; a tile not yet published
    // is waited on alone, within a bound.
    if (d < kRadix) {
        uint32_t excl = 0;
        if (tile > 0) {
            int j = tile - 1;
            int spins = 0;
            for (;;) {
                uint32_t v[kLook];
#pragma unroll
                for (int q = 0; q < kLook; ++q) {
                    // before tile 0: an inclusive prefix of zero
                    uint32_t x = kFlagInc;
                    if (j - q >= 0) x = st[(size_t)(j - q) * kRadix + d];
                    v[q] = x;
                }
                int adv = 0;
                bool done = false;
#pragma unroll
                for (int q = 0; q < kLook; ++q) {
                    if (!done && adv == q && (v[q] & kFlags)) {
                        excl += v[q] & kValMask;
                        if (v[q] & kFlagInc) done = true;
                        else adv = q + 1;
                    }
                }
                if (done) break;
                j -= adv;
                if (adv == 0) {
                    uint32_t x;
                    while (!((x = st[(size_t)j * kRadix + d]) & kFlags) && spins <= kMaxSpin) {
                        ++spins;
                        __nanosleep(64);
                    }
                    if (spins > kMaxSpin) {
                        atomicOr(err, kSortStall);
                        break;
                    }
                    excl += x & kValMask;
                    if (x & kFlagInc) break;
                    --j;
                }
            }
            st[(size_t)tile * kRadix + d] = kFlagInc | (excl + run);
        }
        gdelta[d] = dbase[d] + excl - ts;
    }
    __syncthreads();
#pragma unroll 4
    for (int p = threadIdx.x; p < nv; p += kOsBlock) {
        const uint64_t k = sk[p];
        const uint32_t dd = SYSKEY ? (uint32_t)sd[p] : (uint32_t)(k >> shift) & 0xFFu;
        const uint32_t dst = gdelta[dd] + (uint32_t)p;
        kout[dst] = k;
        vout[dst] = sv[p];
    }
}

template <bool SYSKEY>
__global__ void __launch_bounds__(kOsBlock, kOsMinBlocks) k_onesweep(
    int64_t n, const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
    uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int shift,
    const uint32_t* __restrict__ dbase, uint32_t* status, uint32_t* status_next, uint32_t* tile_ctr,
    const uint32_t* __restrict__ sys, uint32_t* err) {
    constexpr int kWarps = kOsBlock / 32;
    __shared__ uint64_t sk[kOsTile];
    __shared__ uint32_t sv[kOsTile];
    __shared__ uint8_t sd[SYSKEY ? kOsTile : 1];
    __shared__ uint32_t wcnt[kWarps][kRadix];
    __shared__ uint32_t tstart[kRadix];
    __shared__ uint32_t gdelta[kRadix];
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kOsBlock) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int tile = (int)s_tile;
    if ((int64_t)(tile + 1) * kOsTile <= n)
        onesweep_tile<SYSKEY, true>((int)n, tile, kin, vin, kout, vout, shift, dbase, status, status_next,
                                    sys, err, sk, sv, sd, wcnt, tstart, gdelta);
    else
        onesweep_tile<SYSKEY, false>((int)n, tile, kin, vin, kout, vout, shift, dbase, status, status_next,
                                     sys, err, sk, sv, sd, wcnt, tstart, gdelta);
}

// Reorder the particle system into key order and write the FP32 hi/lo
// copies relative to the root centre used by the walk and force kernels.
// If the sort gave up (a look-back wait ran out), the permutation may be
// incomplete: the particles are copied in their current order instead, so
// the system stays whole for the caller's retry.
__global__ void __launch_bounds__(256) k_reorder(
    const DevState* __restrict__ st, int64_t n, const uint32_t* __restrict__ perm, const SysBox* __restrict__ box,
    const uint32_t* __restrict__ sys,
    const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
    const double* __restrict__ vx, const double* __restrict__ vy, const double* __restrict__ vz,
    const double* __restrict__ m, const double* __restrict__ eps, const uint32_t* __restrict__ id,
    double* __restrict__ x2, double* __restrict__ y2, double* __restrict__ z2,
    double* __restrict__ vx2, double* __restrict__ vy2, double* __restrict__ vz2,
    double* __restrict__ m2, double* __restrict__ eps2, uint32_t* __restrict__ id2,
    float4* __restrict__ pf_hi, float4* __restrict__ pf_lo, double* __restrict__ mx2, double* __restrict__ my2,
    double* __restrict__ mz2) {
    const bool sorted = !(st->overflow & kSortInvalid);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const SysBox& b = box[sys ? sys[i] : 0];
        const double c0 = b.c0[0], c1 = b.c0[1], c2 = b.c0[2];
        const uint32_t s = sorted ? perm[i] : (uint32_t)i;
        double px = x[s], py = y[s], pz = z[s], pm = m[s], pe = eps[s];
        x2[i] = px;
        y2[i] = py;
        z2[i] = pz;
        vx2[i] = vx[s];
        vy2[i] = vy[s];
        vz2[i] = vz[s];
        m2[i] = pm;
        eps2[i] = pe;
        id2[i] = id[s];
        double rx = px - c0, ry = py - c1, rz = pz - c2;
        float hx, hy, hz, lx, ly, lz;  // hi/lo parts, converted on the integer pipes
        split_f32(rx, hx, lx);
        split_f32(ry, hy, ly);
        split_f32(rz, hz, lz);
        pf_hi[i] = make_float4(hx, hy, hz, to_f32(pm));
        pf_lo[i] = make_float4(lx, ly, lz, to_f32(pe * pe));
        mx2[i] = __dmul_rn(pm, px);
        my2[i] = __dmul_rn(pm, py);
        mz2[i] = __dmul_rn(pm, pz);
    }
}

}  // namespace

int keys_sort_setup(fdps_ctx* ctx) {
    if (cudaFuncSetAttribute(k_coh_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(CohShared)) !=
        cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, FDPS_ECUDA, "coherent sort set-up failed");
    }
    return FDPS_OK;
}

int keys_and_sort(fdps_tree* t, fdps_psys* ps) {
    fdps_ctx* ctx = t->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t n = ps->n;
    const int c = ps->cur;
    const int ntiles = (int)((n + kOsTile - 1) / kOsTile);
    // the particles are in the order of this tree's last sort (same
    // particle system, same data, moved by the caller since): the coherent
    // sort, with its bucket tables for several systems
    const bool layout = ps->n_sys == 1 || ps->d_cbs;
    const int64_t nbl = ps->n_sys == 1 ? (n + kCohT - 1) / kCohT : ps->coh_nb;
    bool coherent = layout && t->coh_ok && t->coh_ps == ps && t->coh_gen == ps->gen && t->coh_n == n &&
                    n >= 2 * (int64_t)kCohT;
    if (coherent && 3 * nbl + 8 > t->cap_coh) {
        // more buckets than particle tiles (many small systems): grow the
        // counters, except inside a graph capture
        if (ctx->capturing) {
            coherent = false;
        } else {
            dev_free(t->coh_cnt);
            t->cap_coh = 0;
            if (dev_alloc(&t->coh_cnt, 3 * nbl + 8) != cudaSuccess) {
                cudaGetLastError();
                t->coh_cnt = nullptr;
                return set_error(ctx, FDPS_ENOMEM, "coherent-sort counters allocation failed");
            }
            t->cap_coh = 3 * nbl + 8;
        }
    }
    t->coh_ok = layout;
    t->coh_ps = ps;
    t->coh_gen = ps->gen;
    t->coh_n = n;
    t->sort_coherent = coherent;
    if (ps->n_sys == 1) {
        k_box_partial<<<t->box_blocks, kBoxBlock, 0, s>>>(n, ps->x[c], ps->y[c], ps->z[c], t->box_part);
        FDPS_LAUNCH_CHECK(ctx);
        k_box_final<<<1, 32, 0, s>>>(t->box_blocks, t->box_part, t->st, t->sys_box);
        FDPS_LAUNCH_CHECK(ctx);
    } else {
        k_box_seg<<<ps->n_sys, 256, 0, s>>>(ps->d_off, ps->x[c], ps->y[c], ps->z[c], t->sys_box);
        FDPS_LAUNCH_CHECK(ctx);
    }
    if (coherent) {
        CohLayout L;
        L.start = ps->n_sys == 1 ? nullptr : ps->d_cbs;
        L.sys = ps->n_sys == 1 ? nullptr : ps->d_cbsys;
        L.first = ps->n_sys == 1 ? nullptr : ps->d_csfb;
        L.nb = (uint32_t)nbl;
        L.n = n;
        const uint32_t nb = L.nb;
        uint32_t* cnt = t->coh_cnt;
        uint32_t* off = cnt + nb;       // nb + 1
        uint32_t* cur = off + nb + 1;   // nb
        uint32_t* done = cur + nb;
        FDPS_CUDA_TRY(ctx, cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (3 * (size_t)nb + 2), s));
        // the previous sorted keys (keys_b) are the splitters
        k_coh_keys<<<nb, kCohBlock, 0, s>>>(L, ps->x[c], ps->y[c], ps->z[c], t->sys_box, t->keys_b, t->keys_in,
                                             t->coh_bkt, cnt, off, cur, done, &t->st->overflow);
        FDPS_LAUNCH_CHECK(ctx);
        if (t->ev_ok && ctx->profiling && !ctx->capturing) cudaEventRecord(t->ev[1], s);
        k_coh_scatter<<<nb, kCohBlock, 0, s>>>(L, t->keys_in, t->coh_bkt, cur, t->keys_a, t->vals_a,
                                                &t->st->overflow);
        FDPS_LAUNCH_CHECK(ctx);
        k_coh_sort<<<nb, kCohBlock, sizeof(CohShared), s>>>(off, nb, t->keys_a, t->vals_a, t->keys_b, t->vals_b,
                                                             &t->st->overflow);
        FDPS_LAUNCH_CHECK(ctx);
        t->keys_sorted = t->keys_b;
        t->perm = t->vals_b;
        return FDPS_OK;
    }
    // 8 passes over the key; with several systems 2 more, stable, over the
    // system id, so each system's particles end in its own segment in key order
    const int npass = ps->n_sys == 1 ? 8 : 10;
    uint32_t* hist = t->sort_dtot;          // [pass][256] counts, then bases
    uint32_t* tile_ctr = t->sort_dtot + 3072;
    FDPS_CUDA_TRY(ctx, cudaMemsetAsync(t->sort_dtot, 0, sizeof(uint32_t) * 4096, s));
    uint32_t* hist_done = t->sort_dtot + 4000;  // zeroed with the rest above
    k_keys_hist<<<kHistBlocks, kSortBlock, 0, s>>>(n, ps->x[c], ps->y[c], ps->z[c], t->sys_box, ps->d_sys,
                                                   t->keys_in, hist, hist_done);
    FDPS_LAUNCH_CHECK(ctx);
    if (t->ev_ok && ctx->profiling && !ctx->capturing) cudaEventRecord(t->ev[1], s);
    const uint64_t* kin = t->keys_in;
    const uint32_t* vin = nullptr;
    uint64_t* kb[2] = {t->keys_a, t->keys_b};
    uint32_t* vb[2] = {t->vals_a, t->vals_b};
    // [tile][256] look-back words, two buffers: a pass looks back in one and
    // clears the other for the next pass, so only the first needs a memset
    uint32_t* status[2] = {t->sort_hist, t->sort_hist + (size_t)kRadix * ntiles};
    FDPS_CUDA_TRY(ctx, cudaMemsetAsync(status[0], 0, sizeof(uint32_t) * kRadix * (size_t)ntiles, s));
    for (int pass = 0; pass < npass; ++pass) {
        const bool by_sys = pass >= 8;
        const int shift = by_sys ? 8 * (pass - 8) : 8 * pass;
        uint64_t* ko = kb[pass & 1];
        uint32_t* vo = vb[pass & 1];
        uint32_t* st_cur = status[pass & 1];
        uint32_t* st_nxt = status[(pass + 1) & 1];
        if (by_sys)
            k_onesweep<true><<<ntiles, kOsBlock, 0, s>>>(n, kin, vin, ko, vo, shift, hist + pass * kRadix,
                                                           st_cur, st_nxt, tile_ctr + pass, ps->d_sys,
                                                           &t->st->overflow);
        else
            k_onesweep<false><<<ntiles, kOsBlock, 0, s>>>(n, kin, vin, ko, vo, shift, hist + pass * kRadix,
                                                            st_cur, st_nxt, tile_ctr + pass, nullptr,
                                                            &t->st->overflow);
        FDPS_LAUNCH_CHECK(ctx);
        kin = ko;
        vin = vo;
    }
    t->keys_sorted = kb[1];
    t->perm = vb[1];
    return FDPS_OK;
}

// One look-back whose predecessor tile never publishes: the tile counter
// starts at 1, so the single block takes tile 1 and waits on tile 0 until
// its bound runs out.  Every access stays inside the 2-tile buffers.
int selftest_lookback_timeout(fdps_ctx* ctx, uint32_t* flags_out) {
    const int64_t n = 2 * kOsTile;
    uint64_t* keys = nullptr;
    unsigned char* raw = nullptr;
    const size_t bytes = sizeof(uint64_t) * 2 * n + sizeof(uint32_t) * (2 * n + 4 * kRadix + kRadix + 2);
    if (cudaMalloc(&raw, bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, FDPS_ENOMEM, "self-test allocation failed");
    }
    keys = reinterpret_cast<uint64_t*>(raw);
    uint64_t* kout = keys + n;
    uint32_t* vout = reinterpret_cast<uint32_t*>(kout + n);
    uint32_t* status = vout + n;            // 2 tiles x 256
    uint32_t* status_next = status + 2 * kRadix;
    uint32_t* dbase = status_next + 2 * kRadix;  // 256
    uint32_t* ctr = dbase + kRadix;
    uint32_t* err = ctr + 1;
    cudaStream_t s = ctx->stream;
    int rc = FDPS_OK;
    const uint32_t one = 1u;
    if (cudaMemsetAsync(raw, 0, bytes, s) != cudaSuccess ||
        cudaMemcpyAsync(ctr, &one, sizeof(one), cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = set_error(ctx, FDPS_ECUDA, "self-test set-up failed");
    if (!rc) {
        k_onesweep<false><<<1, kOsBlock, 0, s>>>(n, keys, nullptr, kout, vout, 0, dbase, status,
                                                   status_next, ctr, nullptr, err);
        if (cudaGetLastError() != cudaSuccess) rc = set_error(ctx, FDPS_ECUDA, "self-test launch failed");
    }
    uint32_t h = 0;
    if (!rc && (cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess))
        rc = set_error(ctx, FDPS_ECUDA, "self-test readback failed");
    cudaFree(raw);
    *flags_out = h;
    return rc;
}

int reorder_particles(fdps_tree* t, fdps_psys* ps) {
    fdps_ctx* ctx = t->ctx;
    const int c = ps->cur, o = 1 - ps->cur;
    const int64_t n = ps->n;
    int grid = grid_for(n, 256, ctx->sm_count * 16);
    k_reorder<<<grid, 256, 0, ctx->stream>>>(
        t->st, n, t->perm, t->sys_box, ps->d_sys, ps->x[c], ps->y[c], ps->z[c], ps->vx[c], ps->vy[c], ps->vz[c],
        ps->m[c], ps->eps[c], ps->id[c], ps->x[o], ps->y[o], ps->z[o], ps->vx[o], ps->vy[o],
        ps->vz[o], ps->m[o], ps->eps[o], ps->id[o], t->pf_hi, t->pf_lo, t->pmx, t->pmy, t->pmz);
    FDPS_LAUNCH_CHECK(ctx);
    ps->cur = o;
    return FDPS_OK;
}

// ------------------------------------------------- allocation-free variant
//
// fdps_morton_sort_noalloc: root box, Morton keys and the stable sort of one
// particle set with every scratch buffer taken from g_noalloc_scratch, a
// file-scope device array, so the call itself allocates nothing.  It exists
// for callers that may not allocate device memory on their own: hosts such
// as frameworks that hand out every byte of device memory through their own
// pool allocator, and real-time loops that may not take the implicit
// synchronisation and unbounded latency of a cudaMalloc / cudaFree.

namespace {

constexpr int64_t kNoAllocMaxN = int64_t(1) << 18;  // FDPS_NOALLOC_MAX_N
constexpr int kNoAllocBoxBlocks = 256;
constexpr int64_t kNoAllocTiles = kNoAllocMaxN / kSortTile;

constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t kOffState = 0;
constexpr size_t kOffSysBox = align256(kOffState + sizeof(DevState));
constexpr size_t kOffBox = align256(kOffSysBox + sizeof(SysBox));
constexpr size_t kOffHist = align256(kOffBox + sizeof(BoxPartial) * kNoAllocBoxBlocks);
constexpr size_t kOffDtot = align256(kOffHist + sizeof(uint32_t) * kRadix * kNoAllocTiles);
constexpr size_t kOffKeysIn = align256(kOffDtot + sizeof(uint32_t) * kRadix);
constexpr size_t kOffKeysA = align256(kOffKeysIn + sizeof(uint64_t) * kNoAllocMaxN);
constexpr size_t kOffValsA = align256(kOffKeysA + sizeof(uint64_t) * kNoAllocMaxN);
constexpr size_t kNoAllocBytes = align256(kOffValsA + sizeof(uint32_t) * kNoAllocMaxN);

// Held by every device that loads the library, until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// The scratch array's device address per device ordinal, looked up once
// with that device current (in its primary context, the one the runtime
// API uses); written with an atomic store, every writer storing the same
// address.
constexpr int kNoAllocMaxDevices = 64;
std::atomic<unsigned char*> g_noalloc_ptr[kNoAllocMaxDevices] = {};

}  // namespace
}  // namespace fdps

extern "C" int fdps_morton_sort_noalloc(const double* x, const double* y, const double* z,
                                        int64_t n, uint64_t* keys_sorted, uint32_t* perm,
                                        void* stream) {
    using namespace fdps;
    if (!x || !y || !z || !keys_sorted || !perm) return FDPS_EINVAL;
    if (n < 1 || n > kNoAllocMaxN) return FDPS_EINVAL;  // beyond FDPS_NOALLOC_MAX_N
    // an error the calling thread left pending stays the caller's: refuse
    // to run on it rather than clear it
    if (cudaPeekAtLastError() != cudaSuccess) return FDPS_ECUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        cudaGetLastError();
        return FDPS_ECUDA;
    }
    // Once per device, with that device current: the device address of the
    // scratch array (its host-side name is only a stand-in).
    unsigned char* base = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!base) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return FDPS_ECUDA;
        }
        base = static_cast<unsigned char*>(p);
        g_noalloc_ptr[dev].store(base, std::memory_order_release);
    }
    DevState* st = reinterpret_cast<DevState*>(base + kOffState);
    SysBox* sbox = reinterpret_cast<SysBox*>(base + kOffSysBox);
    BoxPartial* box = reinterpret_cast<BoxPartial*>(base + kOffBox);
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + kOffHist);
    uint32_t* dtot = reinterpret_cast<uint32_t*>(base + kOffDtot);
    uint64_t* keys_in = reinterpret_cast<uint64_t*>(base + kOffKeysIn);
    uint64_t* keys_a = reinterpret_cast<uint64_t*>(base + kOffKeysA);
    uint32_t* vals_a = reinterpret_cast<uint32_t*>(base + kOffValsA);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    // The array keeps the previous call's contents.  Every region this call
    // reads is written by an earlier launch of the same call; the state
    // block is cleared anyway, as a defensive measure.
    if (cudaMemsetAsync(st, 0, sizeof(DevState), s) != cudaSuccess) {
        cudaGetLastError();
        return FDPS_ECUDA;
    }
    k_box_partial<<<kNoAllocBoxBlocks, kBoxBlock, 0, s>>>(n, x, y, z, box);
    k_box_final<<<1, 32, 0, s>>>(kNoAllocBoxBlocks, box, st, sbox);
    k_keys<<<ntiles, kSortBlock, 0, s>>>(n, x, y, z, sbox, nullptr, keys_in, hist, ntiles);
    const uint64_t* kin = keys_in;
    const uint32_t* vin = nullptr;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 8 * pass;
        if (pass > 0) k_radix_hist<<<ntiles, kSortBlock, 0, s>>>(n, kin, shift, hist, ntiles);
        k_radix_scan_rows<<<kRadix, 1024, 0, s>>>(hist, ntiles, dtot);
        k_radix_scan_digits<<<1, kRadix, 0, s>>>(dtot);
        // even passes land in the scratch pair, odd ones in the caller's
        // output, so the eighth pass leaves the result there
        uint64_t* ko = (pass & 1) ? keys_sorted : keys_a;
        uint32_t* vo = (pass & 1) ? perm : vals_a;
        k_radix_scatter<<<ntiles, kSortBlock, 0, s>>>(n, kin, vin, ko, vo, shift, hist, dtot, ntiles);
        kin = ko;
        vin = vo;
    }
    if (cudaGetLastError() != cudaSuccess) return FDPS_ECUDA;
    return FDPS_OK;
}
