// integrate.cu -- particle data in and out, input validation, and the
// leapfrog of the paper's N-body example (Sect. 2.2: predict = kick by dt/2
// then drift by dt; correct = kick by dt/2), all in FP64 on the current
// (key-sorted) particle order.
#include <stdlib.h>

#include "fdps_internal.cuh"

namespace fdps {
namespace {

__global__ void __launch_bounds__(256) k_scatter_in(int64_t n, const double* __restrict__ pos,
                                                    const double* __restrict__ vel,
                                                    const double* __restrict__ mass,
                                                    const double* __restrict__ eps, double* x,
                                                    double* y, double* z, double* vx, double* vy,
                                                    double* vz, double* m, double* e, uint32_t* id) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = pos[3 * i];
        y[i] = pos[3 * i + 1];
        z[i] = pos[3 * i + 2];
        vx[i] = vel ? vel[3 * i] : 0.0;
        vy[i] = vel ? vel[3 * i + 1] : 0.0;
        vz[i] = vel ? vel[3 * i + 2] : 0.0;
        m[i] = mass[i];
        e[i] = eps[i];
        id[i] = (uint32_t)i;
    }
}

__global__ void __launch_bounds__(256) k_validate(int64_t n, const double* __restrict__ x,
                                                  const double* __restrict__ y,
                                                  const double* __restrict__ z,
                                                  const double* __restrict__ vx,
                                                  const double* __restrict__ vy,
                                                  const double* __restrict__ vz,
                                                  const double* __restrict__ m,
                                                  const double* __restrict__ e, uint32_t* flag) {
    uint32_t bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!isfinite(x[i]) || !isfinite(y[i]) || !isfinite(z[i])) bad |= 1u;
        if (!isfinite(vx[i]) || !isfinite(vy[i]) || !isfinite(vz[i])) bad |= 2u;
        if (!(m[i] >= 0.0) || !isfinite(m[i])) bad |= 4u;
        if (!(e[i] > 0.0) || !isfinite(e[i])) bad |= 8u;
    }
    bad = __reduce_or_sync(0xFFFFFFFFu, bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicOr(flag, bad);
}

__global__ void __launch_bounds__(256) k_gather_out(int64_t n, const uint32_t* __restrict__ id,
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
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = id[i];
        if (pos) {
            pos[3 * d] = x[i];
            pos[3 * d + 1] = y[i];
            pos[3 * d + 2] = z[i];
        }
        if (vel) {
            vel[3 * d] = vx[i];
            vel[3 * d + 1] = vy[i];
            vel[3 * d + 2] = vz[i];
        }
        if (acc) {
            acc[3 * d] = ax[i];
            acc[3 * d + 1] = ay[i];
            acc[3 * d + 2] = az[i];
        }
        if (pot) pot[d] = phi[i];
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
                      const double* eps) {
    fdps_ctx* ctx = ps->ctx;
    const int c = ps->cur;
    k_scatter_in<<<grid_for(ps->n, 256, ctx->sm_count * 16), 256, 0, ctx->stream>>>(
        ps->n, pos, vel, mass, eps, ps->x[c], ps->y[c], ps->z[c], ps->vx[c], ps->vy[c], ps->vz[c],
        ps->m[c], ps->eps[c], ps->id[c]);
    FDPS_LAUNCH_CHECK(ctx);
    return FDPS_OK;
}

int launch_validate(fdps_psys* ps, uint32_t* bad) {
    fdps_ctx* ctx = ps->ctx;
    const int c = ps->cur;
    FDPS_CUDA_TRY(ctx, cudaMemsetAsync(ps->d_flag, 0, sizeof(uint32_t), ctx->stream));
    k_validate<<<grid_for(ps->n, 256, ctx->sm_count * 16), 256, 0, ctx->stream>>>(
        ps->n, ps->x[c], ps->y[c], ps->z[c], ps->vx[c], ps->vy[c], ps->vz[c], ps->m[c], ps->eps[c],
        ps->d_flag);
    FDPS_LAUNCH_CHECK(ctx);
    FDPS_CUDA_TRY(ctx, cudaMemcpyAsync(bad, ps->d_flag, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                       ctx->stream));
    FDPS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return FDPS_OK;
}

int launch_gather_out(const fdps_psys* ps, double* pos, double* vel, double* acc, double* pot) {
    fdps_ctx* ctx = ps->ctx;
    const int c = ps->cur;
    k_gather_out<<<grid_for(ps->n, 256, ctx->sm_count * 16), 256, 0, ctx->stream>>>(
        ps->n, ps->id[c], ps->x[c], ps->y[c], ps->z[c], ps->vx[c], ps->vy[c], ps->vz[c], ps->ax,
        ps->ay, ps->az, ps->pot, pos, vel, acc, pot);
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
