/* fdps_user_force.cuh -- user interaction laws over the library's lists.
 *
 * FDPS lets its user write the interaction law: the force kernels passed
 * to calcForceAllAndWriteBack take an array of i-particles, an array of
 * j-particles (or superparticles) and the force accumulators (Sect. 2.2).
 * This header is the GPU form of that contract.  The library builds the
 * tree and the interaction lists (fdps_tree_build_lists, or any force
 * calculation) and describes them by a view (fdps_tree_get_view); the
 * template below, compiled into the user's own CUDA code, walks every
 * group's list, stages the list entries in shared memory and calls the
 * user's functors:
 *
 *   struct Force { ...; __device__ void clear(); };
 *   struct Law {
 *     __device__ void operator()(const fdps_user::Epi& i,
 *                                const fdps_user::Epj* j, int nj, Force& f) const;
 *     __device__ void operator()(const fdps_user::Epi& i,
 *                                const fdps_user::Spj* j, int nj, Force& f) const;
 *   };
 *   fdps_tree_view v;  fdps_tree_get_view(tree, ps, &v);
 *   fdps_user::calc_force(v, Law{}, Law{}, out, stream);
 *
 * Each thread owns one i-particle; it calls the functors with tiles of up
 * to 64 particles of opened leaves (EPJ) and up to 32 superparticles (SPJ),
 * which together make the i-particle's group's whole list, in list order.
 * The particle itself is among its EPJ (zero separation): the law decides
 * what that term contributes.  Positions are FP32 relative to the group's
 * centre, formed from hi/lo parts as in the built-in kernel.  out[row] gets
 * the Force of the particle in row `row` of the caller's arrays (cleared,
 * then accumulated by the functors), for every particle.  The work is
 * queued on `stream`; calc_force returns the launch status.
 *
 * The device part of this header (the types and calc_force_body) also
 * compiles under NVRTC, where fdps_user_law_compile builds user laws given
 * as source text at run time.
 */
#pragma once

#ifndef __CUDACC_RTC__
#include <cstdint>
#include <cuda_runtime.h>
#endif

#include "fdps_gpu.h"

namespace fdps_user {

// i-particle: position relative to its group's centre, softening eps^2 and
// the caller's row of the particle
struct Epi {
    float x, y, z, eps2;
    uint32_t row;
};
// particle of an opened leaf, relative to the group centre
struct Epj {
    float x, y, z, m;
};
// superparticle: a cell's centre of mass relative to the group centre, its
// mass and traceless quadrupole about the centre of mass (zero for a
// monopole tree)
struct Spj {
    float x, y, z, m;
    float qxx, qyy, qzz, qxy, qxz, qyz;
};

namespace detail {

constexpr int kWarps = 4;     // warps per block; a warp works on one group at a time
constexpr int kTile = 32;     // list entries per step, one per lane
constexpr int kEpjTile = 64;  // leaf particles per shared tile

__device__ __forceinline__ float4 ld4(const float* p, uint64_t i) {
    return reinterpret_cast<const float4*>(p)[i];
}

// The whole walk over the view's groups, for a block of kWarps warps.
template <class Force, class FEpj, class FSpj>
__device__ __forceinline__ void calc_force_body(const fdps_tree_view& v, const FEpj& f_epj,
                                                const FSpj& f_spj, Force* out) {
    __shared__ Spj s_spj[kWarps][kTile];
    __shared__ Epj s_epj[kWarps][kEpjTile];
    __shared__ uint32_t s_first[kWarps][kTile];
    __shared__ uint32_t s_start[kWarps][kTile];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t g = (int64_t)blockIdx.x * kWarps + w; g < v.n_groups; g += nwarps) {
        const uint32_t gf = v.g_first[g], ni = v.g_count[g];
        const unsigned long long off = v.g_off[g];
        const uint32_t len = v.g_len[g];
        const float4 ch = ld4(v.g_ch, (uint64_t)g), cl = ld4(v.g_cl, (uint64_t)g);
        for (uint32_t ib = 0; ib < ni; ib += 32) {
            const uint32_t i = ib + lane;
            const bool act = i < ni;
            Epi epi{0.f, 0.f, 0.f, 1.f, 0u};
            if (act) {
                const float4 h = ld4(v.pf_hi, gf + i), l = ld4(v.pf_lo, gf + i);
                epi.x = (h.x - ch.x) + (l.x - cl.x);
                epi.y = (h.y - ch.y) + (l.y - cl.y);
                epi.z = (h.z - ch.z) + (l.z - cl.z);
                epi.eps2 = l.w;
                epi.row = v.id[gf + i];
            }
            Force f;
            f.clear();
            for (uint32_t base = 0; base < len; base += kTile) {
                const uint32_t u = base + lane;
                const bool valid = u < len;
                const uint32_t e = valid ? v.pool[off + u] : 0u;
                const bool leaf = valid && (e & v.leaf_tag);
                const bool spj = valid && !leaf;
                const uint32_t node = e & ~v.leaf_tag;
                // superparticles of this step, compacted into the warp's tile
                const uint32_t smask = __ballot_sync(0xFFFFFFFFu, spj);
                if (spj) {
                    const float4 fh = ld4(v.nd_f, 2ull * node), fl = ld4(v.nd_f, 2ull * node + 1);
                    Spj s;
                    s.x = (fh.x - ch.x) + (fl.x - cl.x);
                    s.y = (fh.y - ch.y) + (fl.y - cl.y);
                    s.z = (fh.z - ch.z) + (fl.z - cl.z);
                    s.m = fh.w;
                    s.qxx = s.qyy = s.qzz = s.qxy = s.qxz = s.qyz = 0.f;
                    if (v.quadrupole) {
                        const float4 q0 = ld4(v.nd_fq0, node);
                        const float2 q1 = reinterpret_cast<const float2*>(v.nd_fq1)[node];
                        s.qxx = q0.x;
                        s.qyy = q0.y;
                        s.qzz = q0.z;
                        s.qxy = q0.w;
                        s.qxz = q1.x;
                        s.qyz = q1.y;
                    }
                    s_spj[w][__popc(smask & lt)] = s;
                }
                // opened leaves: particle counts and their offsets in this step
                const uint32_t cnt = leaf ? v.nd_count[node] : 0u;
                uint32_t inc = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                    if (lane >= o) inc += t;
                }
                const uint32_t total = __shfl_sync(0xFFFFFFFFu, inc, 31);
                s_first[w][lane] = leaf ? v.nd_first[node] : 0u;
                s_start[w][lane] = inc - cnt;
                __syncwarp();
                const int nspj = __popc(smask);
                if (act && nspj > 0) f_spj(epi, &s_spj[w][0], nspj, f);
                for (uint32_t c0 = 0; c0 < total; c0 += kEpjTile) {
                    const uint32_t m = total - c0 < (uint32_t)kEpjTile ? total - c0 : (uint32_t)kEpjTile;
                    __syncwarp();
                    for (uint32_t k = lane; k < m; k += 32) {
                        // the owning lane: last lane whose start <= item (lanes
                        // with no particles share the next lane's start)
                        const uint32_t item = c0 + k;
                        int src = 0;
#pragma unroll
                        for (int step = 16; step > 0; step >>= 1)
                            if (s_start[w][src + step] <= item) src += step;
                        const uint32_t p = s_first[w][src] + (item - s_start[w][src]);
                        const float4 h = ld4(v.pf_hi, p), l = ld4(v.pf_lo, p);
                        s_epj[w][k] = Epj{(h.x - ch.x) + (l.x - cl.x), (h.y - ch.y) + (l.y - cl.y),
                                          (h.z - ch.z) + (l.z - cl.z), h.w};
                    }
                    __syncwarp();
                    if (act) f_epj(epi, &s_epj[w][0], (int)m, f);
                }
                __syncwarp();  // the tiles are rewritten in the next step
            }
            if (act) out[epi.row] = f;
        }
    }
}

template <class Force, class FEpj, class FSpj>
__global__ void __launch_bounds__(kWarps * 32)
    calc_force_kernel(fdps_tree_view v, FEpj f_epj, FSpj f_spj, Force* out) {
    calc_force_body<Force>(v, f_epj, f_spj, out);
}

}  // namespace detail

#ifndef __CUDACC_RTC__

// Launch the user laws over every group of the view (see the top of this
// file).  `out` is a device array of v.n Force values.
template <class Force, class FEpj, class FSpj>
cudaError_t calc_force(const fdps_tree_view& v, const FEpj& f_epj, const FSpj& f_spj, Force* out,
                       cudaStream_t stream) {
    if (v.n_groups <= 0) return cudaSuccess;
    int dev = 0, sms = 1, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
             &per_sm, detail::calc_force_kernel<Force, FEpj, FSpj>, detail::kWarps * 32, 0)) != cudaSuccess)
        return e;
    const int64_t need = (v.n_groups + detail::kWarps - 1) / detail::kWarps;
    const int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const int blocks = (int)(need < cap ? need : cap);
    detail::calc_force_kernel<Force, FEpj, FSpj>
        <<<blocks, detail::kWarps * 32, 0, stream>>>(v, f_epj, f_spj, out);
    return cudaGetLastError();
}
#endif  // __CUDACC_RTC__

}  // namespace fdps_user
