// integrate.cu -- particle data in and out, input validation, and the
// leapfrog of the paper's N-body example (Sect. 2.2: predict = kick by dt/2
// then drift by dt; correct = kick by dt/2), all in FP64 on the current
// (key-sorted) particle order.
#include <stdlib.h>

#include "fdps_internal.cuh"

namespace fdps {
namespace {

// The input rules as bit tests (FP64 compares run on a narrow pipe on this
// part): finite = exponent field not all ones; mass >= 0 holds for +0, -0
// and positive values; eps > 0 for positive nonzero values.
__device__ __forceinline__ bool finite64(double v) {
    return ((__double_as_longlong(v) >> 52) & 0x7FF) != 0x7FF;
}
__device__ __forceinline__ bool nonneg64(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) == 0 || b == 0x8000000000000000ull;
}
__device__ __forceinline__ bool positive64(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) == 0 && b != 0;
}

constexpr int kIoTile = 256;  // particles per block and round of the in/out kernels

// [n][3] rows base .. base + m of a caller array into s[3 m] (flat, so that
// a warp's loads are contiguous: this matters when the array is host memory
// read over the CPU-GPU link).
__device__ __forceinline__ void load_rows3(const double* __restrict__ a, int64_t base, int m, double* s) {
    for (int k = threadIdx.x; k < 3 * m; k += kIoTile) s[k] = a[3 * base + k];
}
__device__ __forceinline__ void store_rows3(double* a, int64_t base, int m, const double* s) {
    for (int k = threadIdx.x; k < 3 * m; k += kIoTile) a[3 * base + k] = s[k];
}

// Caller-order input arrays (device memory, or host memory the device can
// read) into the structure-of-arrays buffers, checked on the way: flag bit
// 1 a non-finite position, 2 a non-finite velocity, 4 a negative or
// non-finite mass, 8 a non-positive or non-finite softening.  Caller row i
// goes to position inv[i] (the order the buffers already hold; the caller
// arrays are still read contiguously), or with inv null to position i with
// id[i] = i.  With inv, a record buffer rec (64 bytes a particle) takes the
// particle's eight values as one record at position inv[i] (whole 32-byte
// sectors, where scattered 8-byte writes into eight arrays would each
// rewrite part of a sector); k_rec_split then fills the arrays in order.
__global__ void __launch_bounds__(kIoTile) k_scatter_in(int64_t n, const double* __restrict__ pos,
                                                        const double* __restrict__ vel,
                                                        const double* __restrict__ mass,
                                                        const double* __restrict__ eps, double* x,
                                                        double* y, double* z, double* vx, double* vy,
                                                        double* vz, double* m, double* e, uint32_t* id,
                                                        const uint32_t* __restrict__ inv, double2* rec,
                                                        uint32_t* flag) {
    __shared__ double s_p[3 * kIoTile], s_v[3 * kIoTile];
    uint32_t bad = 0;
    for (int64_t base = (int64_t)blockIdx.x * kIoTile; base < n; base += (int64_t)gridDim.x * kIoTile) {
        const int cnt = n - base < kIoTile ? (int)(n - base) : kIoTile;
        load_rows3(pos, base, cnt, s_p);
        if (vel) load_rows3(vel, base, cnt, s_v);
        __syncthreads();
        const int t = threadIdx.x;
        if (t < cnt) {
            const int64_t i = base + t;
            const double px = s_p[3 * t], py = s_p[3 * t + 1], pz = s_p[3 * t + 2];
            const double ux = vel ? s_v[3 * t] : 0.0, uy = vel ? s_v[3 * t + 1] : 0.0,
                         uz = vel ? s_v[3 * t + 2] : 0.0;
            const double mi = mass[i], ei = eps[i];
            bad |= (finite64(px) && finite64(py) && finite64(pz)) ? 0u : 1u;
            bad |= (finite64(ux) && finite64(uy) && finite64(uz)) ? 0u : 2u;
            bad |= (finite64(mi) && nonneg64(mi)) ? 0u : 4u;
            bad |= (finite64(ei) && positive64(ei)) ? 0u : 8u;
            const int64_t d = inv ? (int64_t)inv[i] : i;
            if (rec) {
                double2* r = rec + 4 * d;
                r[0] = make_double2(px, py);
                r[1] = make_double2(pz, ux);
                r[2] = make_double2(uy, uz);
                r[3] = make_double2(mi, ei);
            } else {
                x[d] = px;
                y[d] = py;
                z[d] = pz;
                vx[d] = ux;
                vy[d] = uy;
                vz[d] = uz;
                m[d] = mi;
                e[d] = ei;
            }
            if (!inv) id[i] = (uint32_t)i;
        }
        __syncthreads();  // the tiles are rewritten next round
    }
    bad = __reduce_or_sync(0xFFFFFFFFu, bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicOr(flag, bad);
}

// Records (x, y, z, vx, vy, vz, m, eps) in position order into the arrays.
__global__ void __launch_bounds__(256) k_rec_split(int64_t n, const double2* __restrict__ rec, double* x,
                                                   double* y, double* z, double* vx, double* vy, double* vz,
                                                   double* m, double* e) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = rec[4 * j], b = rec[4 * j + 1], c = rec[4 * j + 2], d = rec[4 * j + 3];
        x[j] = a.x;
        y[j] = a.y;
        z[j] = b.x;
        vx[j] = b.y;
        vy[j] = c.x;
        vz[j] = c.y;
        m[j] = d.x;
        e[j] = d.y;
    }
}

// Inverse of the current order: inv[caller index] = position.
__global__ void __launch_bounds__(256) k_invert(int64_t n, const uint32_t* __restrict__ id,
                                                uint32_t* __restrict__ inv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        inv[id[i]] = (uint32_t)i;
}

// Results in the caller's order: a block takes kIoTile consecutive caller
// indices j, reads each from position inv[j] and writes the rows out
// contiguously (through shared memory for the [n][3] arrays).
__global__ void __launch_bounds__(kIoTile) k_gather_out(int64_t n, const uint32_t* __restrict__ inv,
                                                        const double* __restrict__ x,
                                                        const double* __restrict__ y,
                                                        const double* __restrict__ z,
                                                        const double* __restrict__ vx,
                                                        const double* __restrict__ vy,
                                                        const double* __restrict__ vz,
                                                        const double* __restrict__ ax,
                                                        const double* __restrict__ ay,
                                                        const double* __restrict__ az,
                                                        const double* __restrict__ phi, double* pos,
                                                        double* vel, double* acc, double* pot) {
    __shared__ double s_t[3 * kIoTile];
    for (int64_t base = (int64_t)blockIdx.x * kIoTile; base < n; base += (int64_t)gridDim.x * kIoTile) {
        const int cnt = n - base < kIoTile ? (int)(n - base) : kIoTile;
        const int t = threadIdx.x;
        const int64_t s = t < cnt ? (int64_t)inv[base + t] : 0;
        const double* src[3][3] = {{x, y, z}, {vx, vy, vz}, {ax, ay, az}};
        double* dst[3] = {pos, vel, acc};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!dst[a]) continue;
            if (t < cnt) {
                s_t[3 * t] = src[a][0][s];
                s_t[3 * t + 1] = src[a][1][s];
                s_t[3 * t + 2] = src[a][2][s];
            }
            __syncthreads();
            store_rows3(dst[a], base, cnt, s_t);
            __syncthreads();
        }
        if (pot && t < cnt) pot[base + t] = phi[s];
    }
}

__global__ void __launch_bounds__(256) k_kick(int64_t n, double h, double* vx, double* vy, double* vz,
                                              const double* __restrict__ ax,
                                              const double* __restrict__ ay,
                                              const double* __restrict__ az) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        vx[i] += h * ax[i];
        vy[i] += h * ay[i];
        vz[i] += h * az[i];
    }
}

// The first half-kick and the drift of a step in one pass (the same two
// updates per particle, in the same order, as k_kick then k_drift).
__global__ void __launch_bounds__(256) k_kick_drift(int64_t n, double h, double dt, double* x, double* y,
                                                    double* z, double* vx, double* vy, double* vz,
                                                    const double* __restrict__ ax,
                                                    const double* __restrict__ ay,
                                                    const double* __restrict__ az) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double ux = vx[i] + h * ax[i], uy = vy[i] + h * ay[i], uz = vz[i] + h * az[i];
        vx[i] = ux;
        vy[i] = uy;
        vz[i] = uz;
        x[i] += dt * ux;
        y[i] += dt * uy;
        z[i] += dt * uz;
    }
}
__global__ void __launch_bounds__(256) k_drift(int64_t n, double dt, double* x, double* y, double* z,
                                               const double* __restrict__ vx,
                                               const double* __restrict__ vy,
                                               const double* __restrict__ vz) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += dt * vx[i];
        y[i] += dt * vy[i];
        z[i] += dt * vz[i];
    }
}

// Per-block partial sums of m v^2 / 2 and m phi / 2, combined on one block.
__global__ void __launch_bounds__(256) k_energy_partial(int64_t n, const double* __restrict__ vx,
                                                        const double* __restrict__ vy,
                                                        const double* __restrict__ vz,
                                                        const double* __restrict__ m,
                                                        const double* __restrict__ phi,
                                                        double* part) {
    double ek = 0.0, ep = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        ek += 0.5 * m[i] * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]);
        ep += 0.5 * m[i] * phi[i];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ek += __shfl_xor_sync(0xFFFFFFFFu, ek, off);
        ep += __shfl_xor_sync(0xFFFFFFFFu, ep, off);
    }
    __shared__ double s[2][8];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s[0][w] = ek;
        s[1][w] = ep;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a += s[0][k];
            b += s[1][k];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void k_energy_final(int nb, double* part) {
    if (threadIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nb; ++k) {
        a += part[2 * k];
        b += part[2 * k + 1];
    }
    part[2 * nb] = a;
    part[2 * nb + 1] = b;
}

constexpr int kEnergyBlocks = 512;

__global__ void __launch_bounds__(256) k_sys_index(const int64_t* __restrict__ off, uint32_t* sys) {
    const int64_t a = off[blockIdx.x], b = off[blockIdx.x + 1];
    for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) sys[i] = blockIdx.x;
}

// Kinetic and potential energy of each system: one block per system.
__global__ void __launch_bounds__(256) k_energy_seg(const int64_t* __restrict__ off,
                                                    const double* __restrict__ vx,
                                                    const double* __restrict__ vy,
                                                    const double* __restrict__ vz,
                                                    const double* __restrict__ m,
                                                    const double* __restrict__ phi, double* out) {
    const int64_t a = off[blockIdx.x], b = off[blockIdx.x + 1];
    double ek = 0.0, ep = 0.0;
    for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
        ek += 0.5 * m[i] * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]);
        ep += 0.5 * m[i] * phi[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ek += __shfl_xor_sync(0xFFFFFFFFu, ek, o);
        ep += __shfl_xor_sync(0xFFFFFFFFu, ep, o);
    }
    __shared__ double s[2][8];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s[0][w] = ek;
        s[1][w] = ep;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            x += s[0][k];
            y += s[1][k];
        }
        out[2 * blockIdx.x] = x;
        out[2 * blockIdx.x + 1] = y;
    }
}

// The second kick of a captured step; skipped when that step's force
// calculation overflowed a buffer (the host then redoes the force and kick).
__global__ void __launch_bounds__(256) k_kick_guarded(int64_t n, double h, double* vx, double* vy,
                                                      double* vz, const double* __restrict__ ax,
                                                      const double* __restrict__ ay,
                                                      const double* __restrict__ az,
                                                      const uint32_t* __restrict__ flags,
                                                      uint32_t mask) {
    if (*flags & mask) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        vx[i] += h * ax[i];
        vy[i] += h * ay[i];
        vz[i] += h * az[i];
    }
}

}  // namespace

int launch_kick_guarded(fdps_psys* ps, double dt_half, const uint32_t* flags, uint32_t mask) {
    fdps_ctx* ctx = ps->ctx;
    const int c = ps->cur;
    k_kick_guarded<<<grid_for(ps->n, 256, ctx->sm_count * 16), 256, 0, ctx->stream>>>(
        ps->n, dt_half, ps->vx[c], ps->vy[c], ps->vz[c], ps->ax, ps->ay, ps->az, flags, mask);
    FDPS_LAUNCH_CHECK(ctx);
    return FDPS_OK;
}

int launch_sys_index(fdps_psys* ps) {
    fdps_ctx* ctx = ps->ctx;
    k_sys_index<<<ps->n_sys, 256, 0, ctx->stream>>>(ps->d_off, ps->d_sys);
    FDPS_LAUNCH_CHECK(ctx);
    return FDPS_OK;
}

int launch_energy_systems(fdps_psys* ps, double* kin, double* pot) {
    fdps_ctx* ctx = ps->ctx;
    const int c = ps->cur;
    const int64_t S = ps->n_sys;
    if (ps->n_sys == 1) return launch_energy(ps, kin, pot);
    k_energy_seg<<<ps->n_sys, 256, 0, ctx->stream>>>(ps->d_off, ps->vx[c], ps->vy[c], ps->vz[c],
                                                    ps->m[c], ps->pot, ps->d_sys_red);
    FDPS_LAUNCH_CHECK(ctx);
    double* h = (double*)malloc(sizeof(double) * 2 * S);
    if (!h) return set_error(ctx, FDPS_ENOMEM, "host allocation failed");
    cudaError_t e = cudaMemcpyAsync(h, ps->d_sys_red, sizeof(double) * 2 * S, cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    if (!e)
        for (int64_t k = 0; k < S; ++k) {
            kin[k] = h[2 * k];
            pot[k] = h[2 * k + 1];
        }
    free(h);
    if (e) return set_error(ctx, FDPS_ECUDA, "energy readback failed: %s", cudaGetErrorString(e));
    return FDPS_OK;
}

int energy_scratch_doubles() { return 2 * kEnergyBlocks + 2; }

int launch_scatter_in(fdps_psys* ps, const double* pos, const double* vel, const double* mass,
                      const double* eps, bool keep_order, uint32_t* bad) {
    fdps_ctx* ctx = ps->ctx;
    if (!keep_order) ps->cur = 0;
    const int c = ps->cur;
    if (keep_order) {
        if (!ps->inv && dev_alloc(&ps->inv, ps->n) != cudaSuccess) {
            cudaGetLastError();
            ps->inv = nullptr;
            return set_error(ctx, FDPS_ENOMEM, "inverse-order allocation failed");
        }
        k_invert<<<grid_for(ps->n, 256, ctx->sm_count * 16), 256, 0, ctx->stream>>>(ps->n, ps->id[c], ps->inv);
        FDPS_LAUNCH_CHECK(ctx);
        // without the record buffer the values are written straight into
        // the arrays (scattered 8-byte writes, slower)
        if (!ps->rec && dev_alloc(&ps->rec, 8 * ps->n) != cudaSuccess) {
            cudaGetLastError();
            ps->rec = nullptr;
        }
    }
    double2* rec = keep_order ? reinterpret_cast<double2*>(ps->rec) : nullptr;
    FDPS_CUDA_TRY(ctx, cudaMemsetAsync(ps->d_flag, 0, sizeof(uint32_t), ctx->stream));
    k_scatter_in<<<grid_for(ps->n, kIoTile, ctx->sm_count * 8), kIoTile, 0, ctx->stream>>>(
        ps->n, pos, vel, mass, eps, ps->x[c], ps->y[c], ps->z[c], ps->vx[c], ps->vy[c], ps->vz[c],
        ps->m[c], ps->eps[c], ps->id[c], keep_order ? ps->inv : nullptr, rec, ps->d_flag);
    FDPS_LAUNCH_CHECK(ctx);
    if (rec) {
        k_rec_split<<<grid_for(ps->n, 256, ctx->sm_count * 16), 256, 0, ctx->stream>>>(
            ps->n, rec, ps->x[c], ps->y[c], ps->z[c], ps->vx[c], ps->vy[c], ps->vz[c], ps->m[c], ps->eps[c]);
        FDPS_LAUNCH_CHECK(ctx);
    }
    FDPS_CUDA_TRY(ctx, cudaMemcpyAsync(bad, ps->d_flag, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                       ctx->stream));
    FDPS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return FDPS_OK;
}

int launch_gather_out(fdps_psys* ps, double* pos, double* vel, double* acc, double* pot) {
    fdps_ctx* ctx = ps->ctx;
    const int c = ps->cur;
    if (!ps->inv && dev_alloc(&ps->inv, ps->n) != cudaSuccess) {
        cudaGetLastError();
        ps->inv = nullptr;
        return set_error(ctx, FDPS_ENOMEM, "inverse-order allocation failed");
    }
    const int grid = grid_for(ps->n, 256, ctx->sm_count * 16);
    k_invert<<<grid, 256, 0, ctx->stream>>>(ps->n, ps->id[c], ps->inv);
    FDPS_LAUNCH_CHECK(ctx);
    k_gather_out<<<grid_for(ps->n, kIoTile, ctx->sm_count * 8), kIoTile, 0, ctx->stream>>>(ps->n, ps->inv, ps->x[c], ps->y[c], ps->z[c], ps->vx[c],
                                                ps->vy[c], ps->vz[c], ps->ax, ps->ay, ps->az, ps->pot, pos, vel,
                                                acc, pot);
    FDPS_LAUNCH_CHECK(ctx);
    return FDPS_OK;
}

int launch_kick(fdps_psys* ps, double dt_half) {
    fdps_ctx* ctx = ps->ctx;
    const int c = ps->cur;
    k_kick<<<grid_for(ps->n, 256, ctx->sm_count * 16), 256, 0, ctx->stream>>>(
        ps->n, dt_half, ps->vx[c], ps->vy[c], ps->vz[c], ps->ax, ps->ay, ps->az);
    FDPS_LAUNCH_CHECK(ctx);
    return FDPS_OK;
}

int launch_kick_drift(fdps_psys* ps, double dt_half, double dt) {
    fdps_ctx* ctx = ps->ctx;
    const int c = ps->cur;
    k_kick_drift<<<grid_for(ps->n, 256, ctx->sm_count * 16), 256, 0, ctx->stream>>>(
        ps->n, dt_half, dt, ps->x[c], ps->y[c], ps->z[c], ps->vx[c], ps->vy[c], ps->vz[c], ps->ax, ps->ay,
        ps->az);
    FDPS_LAUNCH_CHECK(ctx);
    return FDPS_OK;
}
int launch_drift(fdps_psys* ps, double dt) {
    fdps_ctx* ctx = ps->ctx;
    const int c = ps->cur;
    k_drift<<<grid_for(ps->n, 256, ctx->sm_count * 16), 256, 0, ctx->stream>>>(
        ps->n, dt, ps->x[c], ps->y[c], ps->z[c], ps->vx[c], ps->vy[c], ps->vz[c]);
    FDPS_LAUNCH_CHECK(ctx);
    return FDPS_OK;
}

int launch_energy(fdps_psys* ps, double* kin, double* pot) {
    fdps_ctx* ctx = ps->ctx;
    const int c = ps->cur;
    k_energy_partial<<<kEnergyBlocks, 256, 0, ctx->stream>>>(ps->n, ps->vx[c], ps->vy[c], ps->vz[c],
                                                             ps->m[c], ps->pot, ps->d_red);
    FDPS_LAUNCH_CHECK(ctx);
    k_energy_final<<<1, 32, 0, ctx->stream>>>(kEnergyBlocks, ps->d_red);
    FDPS_LAUNCH_CHECK(ctx);
    double h[2];
    FDPS_CUDA_TRY(ctx, cudaMemcpyAsync(h, ps->d_red + 2 * kEnergyBlocks, sizeof(h),
                                       cudaMemcpyDeviceToHost, ctx->stream));
    FDPS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    *kin = h[0];
    *pot = h[1];
    return FDPS_OK;
}

}  // namespace fdps
