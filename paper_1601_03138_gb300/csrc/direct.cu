// direct.cu -- direct summation for a sample of particles, the exact
// reference of the tree force (Eq. ParticleParticleNbody summed over every
// other particle of the same system, softening of the receiving particle).
//
// Used to measure the tree's force error on the GPU and to choose the
// opening angle for an error target.  Arithmetic: positions as FP32 hi/lo
// parts relative to a common origin, so that separations keep about 48
// bits; each pair in FP32 with MUFU rsqrt; per-tile FP32 sums added into
// Kahan-compensated totals, finished in FP64.  Particle i's own term is
// skipped.
#include "fdps_internal.cuh"

namespace fdps {
namespace {

constexpr int kDB = 128;  // sampled i-particles per block
constexpr int kDT = 256;  // j-particles per shared tile

__global__ void __launch_bounds__(256) k_direct_prep(int64_t n, const double* __restrict__ x,
                                                     const double* __restrict__ y,
                                                     const double* __restrict__ z,
                                                     const double* __restrict__ m,
                                                     const double* __restrict__ eps, double ox,
                                                     double oy, double oz, float4* __restrict__ hi,
                                                     float4* __restrict__ lo) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double rx = x[i] - ox, ry = y[i] - oy, rz = z[i] - oz;
        const float hx = __double2float_rn(rx), hy = __double2float_rn(ry), hz = __double2float_rn(rz);
        hi[i] = make_float4(hx, hy, hz, __double2float_rn(m[i]));
        lo[i] = make_float4(__double2float_rn(rx - (double)hx), __double2float_rn(ry - (double)hy),
                            __double2float_rn(rz - (double)hz), __double2float_rn(eps[i] * eps[i]));
    }
}

__global__ void k_invert_id(int64_t n, const uint32_t* __restrict__ id, uint32_t* __restrict__ inv) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        inv[id[p]] = (uint32_t)p;
}

struct Comp4 {
    float s[4], c[4];
    __device__ __forceinline__ void add(int k, float v) {
        const float y = v - c[k];
        const float t = s[k] + y;
        c[k] = (t - s[k]) - y;
        s[k] = t;
    }
};

// one pair: (dx, dy, dz) from i to j, adds m/r^3 d and -m/r
__device__ __forceinline__ void pair(const float4 ih, const float4 il, const float4 jh, const float4 jl,
                                     float e2, float& ax, float& ay, float& az, float& pp) {
    const float dx = (jh.x - ih.x) + (jl.x - il.x);
    const float dy = (jh.y - ih.y) + (jl.y - il.y);
    const float dz = (jh.z - ih.z) + (jl.z - il.z);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, e2)));
    const float ri = rsqrtf(r2);
    const float mri = jh.w * ri;
    const float mri3 = mri * ri * ri;
    ax = fmaf(mri3, dx, ax);
    ay = fmaf(mri3, dy, ay);
    az = fmaf(mri3, dz, az);
    pp -= mri;
}

// One system: block (x: 128 sampled particles, y: one slice of the j range),
// j-particles staged in shared tiles; partial sums per slice in FP64.
__global__ void __launch_bounds__(kDB) k_direct_tiled(int64_t n, int64_t ns, const uint32_t* __restrict__ inv,
                                                      const int64_t* __restrict__ rows,
                                                      const float4* __restrict__ hi,
                                                      const float4* __restrict__ lo, int64_t jper,
                                                      double* __restrict__ part) {
    __shared__ float4 s_h[kDT], s_l[kDT];
    const int t = threadIdx.x;
    const int64_t s = blockIdx.x * (int64_t)kDB + t;
    const bool valid = s < ns;
    const int64_t p = valid ? (int64_t)inv[rows[s]] : -1;
    const float4 ih = valid ? hi[p] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 il = valid ? lo[p] : make_float4(0.f, 0.f, 0.f, 1.f);
    const int64_t j0 = blockIdx.y * jper;
    const int64_t j1 = j0 + jper < n ? j0 + jper : n;
    Comp4 acc;
#pragma unroll
    for (int k = 0; k < 4; ++k) acc.s[k] = acc.c[k] = 0.f;
    for (int64_t jt = j0; jt < j1; jt += kDT) {
        const int m = j1 - jt < kDT ? (int)(j1 - jt) : kDT;
        __syncthreads();
        for (int k = t; k < m; k += kDB) {
            s_h[k] = hi[jt + k];
            s_l[k] = lo[jt + k];
        }
        __syncthreads();
        float ax = 0.f, ay = 0.f, az = 0.f, pp = 0.f;
        for (int k = 0; k < m; ++k) {
            if (jt + k == p) continue;  // no self term
            pair(ih, il, s_h[k], s_l[k], il.w, ax, ay, az, pp);
        }
        acc.add(0, ax);
        acc.add(1, ay);
        acc.add(2, az);
        acc.add(3, pp);
    }
    if (valid)
#pragma unroll
        for (int k = 0; k < 4; ++k)
            part[((int64_t)blockIdx.y * ns + s) * 4 + k] = (double)acc.s[k] - (double)acc.c[k];
}

// Several systems: each sampled particle sums over its own system's range.
__global__ void __launch_bounds__(kDB) k_direct_systems(int64_t ns, const uint32_t* __restrict__ inv,
                                                        const int64_t* __restrict__ rows,
                                                        const uint32_t* __restrict__ sys,
                                                        const int64_t* __restrict__ off,
                                                        const float4* __restrict__ hi,
                                                        const float4* __restrict__ lo,
                                                        double* __restrict__ part) {
    const int64_t s = blockIdx.x * (int64_t)kDB + threadIdx.x;
    if (s >= ns) return;
    const int64_t p = inv[rows[s]];
    const float4 ih = hi[p], il = lo[p];
    const uint32_t k = sys[p];
    Comp4 acc;
#pragma unroll
    for (int c = 0; c < 4; ++c) acc.s[c] = acc.c[c] = 0.f;
    for (int64_t jt = off[k]; jt < off[k + 1]; jt += kDT) {
        const int64_t je = jt + kDT < off[k + 1] ? jt + kDT : off[k + 1];
        float ax = 0.f, ay = 0.f, az = 0.f, pp = 0.f;
        for (int64_t j = jt; j < je; ++j) {
            if (j == p) continue;
            pair(ih, il, hi[j], lo[j], il.w, ax, ay, az, pp);
        }
        acc.add(0, ax);
        acc.add(1, ay);
        acc.add(2, az);
        acc.add(3, pp);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) part[s * 4 + c] = (double)acc.s[c] - (double)acc.c[c];
}

__global__ void k_direct_final(int64_t ns, int js, const double* __restrict__ part, double* __restrict__ out) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns;
         s += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double v = 0.0;
            for (int y = 0; y < js; ++y) v += part[((int64_t)y * ns + s) * 4 + k];
            out[s * 4 + k] = v;
        }
}

// Tree results (acceleration, potential) at the sampled rows.
__global__ void k_gather_rows(int64_t ns, const uint32_t* __restrict__ inv, const int64_t* __restrict__ rows,
                              const double* __restrict__ ax, const double* __restrict__ ay,
                              const double* __restrict__ az, const double* __restrict__ pot,
                              double* __restrict__ out) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns;
         s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = inv[rows[s]];
        out[s * 4 + 0] = ax[p];
        out[s * 4 + 1] = ay[p];
        out[s * 4 + 2] = az[p];
        out[s * 4 + 3] = pot[p];
    }
}

}  // namespace

// Scratch of a sample: inverse of the id map, FP32 hi/lo copies (direct
// sums only), partial sums.  All device memory, freed by the caller with
// free_sample_scratch.
struct SampleScratch {
    uint32_t* inv = nullptr;
    float4* hi = nullptr;
    float4* lo = nullptr;
    double* part = nullptr;
};

static void free_sample_scratch(SampleScratch& sc) {
    cudaFree(sc.inv);
    cudaFree(sc.hi);
    cudaFree(sc.lo);
    cudaFree(sc.part);
    sc = SampleScratch{};
}

static int invert_ids(fdps_psys* ps, SampleScratch& sc) {
    fdps_ctx* ctx = ps->ctx;
    if (!sc.inv && cudaMalloc(&sc.inv, sizeof(uint32_t) * (size_t)ps->n) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, FDPS_ENOMEM, "sample scratch allocation failed");
    }
    k_invert_id<<<grid_for(ps->n, 256, 4 * ctx->sm_count), 256, 0, ctx->stream>>>(ps->n, ps->id[ps->cur], sc.inv);
    FDPS_LAUNCH_CHECK(ctx);
    return FDPS_OK;
}

int direct_sample_device(fdps_psys* ps, int64_t ns, const int64_t* d_rows, double* d_out4) {
    fdps_ctx* ctx = ps->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t n = ps->n;
    const int c = ps->cur;
    SampleScratch sc;
    int rc = invert_ids(ps, sc);
    const bool one = ps->n_sys == 1;
    // slices of the j range: enough blocks to fill the GPU
    const int64_t bx = (ns + kDB - 1) / kDB;
    int js = one ? (int)((4 * ctx->sm_count + bx - 1) / bx) : 1;
    if (js < 1) js = 1;
    if (js > 1024) js = 1024;
    if (!rc && (cudaMalloc(&sc.hi, sizeof(float4) * (size_t)n) != cudaSuccess ||
                cudaMalloc(&sc.lo, sizeof(float4) * (size_t)n) != cudaSuccess ||
                cudaMalloc(&sc.part, sizeof(double) * 4 * (size_t)ns * js) != cudaSuccess)) {
        cudaGetLastError();
        rc = set_error(ctx, FDPS_ENOMEM, "sample scratch allocation failed");
    }
    if (!rc) {
        // origin: the first particle's position (separations are what count)
        double o[3];
        if (cudaMemcpyAsync(&o[0], ps->x[c], 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&o[1], ps->y[c], 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&o[2], ps->z[c], 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = set_error(ctx, FDPS_ECUDA, "reading the origin failed");
        if (!rc) {
            k_direct_prep<<<grid_for(n, 256, 4 * ctx->sm_count), 256, 0, s>>>(
                n, ps->x[c], ps->y[c], ps->z[c], ps->m[c], ps->eps[c], o[0], o[1], o[2], sc.hi, sc.lo);
            FDPS_LAUNCH_CHECK(ctx);
            if (one) {
                const int64_t jper = (n + js - 1) / js;
                k_direct_tiled<<<dim3((unsigned)bx, (unsigned)js), kDB, 0, s>>>(n, ns, sc.inv, d_rows, sc.hi,
                                                                              sc.lo, jper, sc.part);
            } else {
                k_direct_systems<<<(unsigned)bx, kDB, 0, s>>>(ns, sc.inv, d_rows, ps->d_sys, ps->d_off, sc.hi,
                                                              sc.lo, sc.part);
            }
            FDPS_LAUNCH_CHECK(ctx);
            k_direct_final<<<grid_for(ns, 256, 1024), 256, 0, s>>>(ns, js, sc.part, d_out4);
            FDPS_LAUNCH_CHECK(ctx);
            if (cudaStreamSynchronize(s) != cudaSuccess) rc = set_error(ctx, FDPS_ECUDA, "direct sum failed");
        }
    }
    free_sample_scratch(sc);
    return rc;
}

int gather_rows_device(fdps_psys* ps, int64_t ns, const int64_t* d_rows, double* d_out4) {
    fdps_ctx* ctx = ps->ctx;
    SampleScratch sc;
    int rc = invert_ids(ps, sc);
    if (!rc) {
        k_gather_rows<<<grid_for(ns, 256, 1024), 256, 0, ctx->stream>>>(ns, sc.inv, d_rows, ps->ax, ps->ay,
                                                                       ps->az, ps->pot, d_out4);
        FDPS_LAUNCH_CHECK(ctx);
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = set_error(ctx, FDPS_ECUDA, "gather failed");
    }
    free_sample_scratch(sc);
    return rc;
}

}  // namespace fdps
