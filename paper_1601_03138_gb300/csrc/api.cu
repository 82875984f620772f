// api.cu -- the C ABI of include/fdps_gpu.h: handles, buffer management and
// the force-calculation pipeline of calcForceAllAndWriteBack (Sect. 2.2 and
// Sect. 3.2 of Iwasawa et al. 2016, on one GPU: local tree = global tree).
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "fdps_internal.cuh"

namespace fdps {
int walk_blocks(fdps_ctx* ctx);
int walk_warps_per_block();
unsigned long long walk_chunk();
int launch_walk(fdps_tree* t, const uint32_t* sys, int blocks);
int energy_scratch_doubles();
}  // namespace fdps

using namespace fdps;

namespace {

constexpr int kSortTile = 2048;
static_assert(kSortTile == kBuildTile, "one tile count sizes the sort and build scratch");

void free_particles(fdps_tree* t) {
    dev_free(t->keys_in);
    dev_free(t->keys_a);
    dev_free(t->keys_b);
    dev_free(t->vals_a);
    dev_free(t->vals_b);
    dev_free(t->pf_hi);
    dev_free(t->pf_lo);
    dev_free(t->pmx);
    dev_free(t->pmy);
    dev_free(t->pmz);
    dev_free(t->head);
    dev_free(t->sort_hist);
    dev_free(t->bt_count);
    dev_free(t->coh_bkt);
    dev_free(t->coh_cnt);
    t->cap_coh = 0;
    t->coh_ok = false;  // the last sorted keys are gone
    t->cap_n = 0;
    t->cap_tiles = 0;
}

int ensure_particles(fdps_tree* t, int64_t n) {
    if (n <= t->cap_n) return FDPS_OK;
    free_particles(t);
    const int64_t tiles = (n + kSortTile - 1) / kSortTile;
    bool ok = dev_alloc(&t->keys_in, n) == cudaSuccess && dev_alloc(&t->keys_a, n) == cudaSuccess &&
              dev_alloc(&t->keys_b, n) == cudaSuccess && dev_alloc(&t->vals_a, n) == cudaSuccess &&
              dev_alloc(&t->vals_b, n) == cudaSuccess && dev_alloc(&t->pf_hi, n) == cudaSuccess &&
              dev_alloc(&t->pf_lo, n) == cudaSuccess && dev_alloc(&t->head, n) == cudaSuccess &&
              dev_alloc(&t->pmx, n) == cudaSuccess && dev_alloc(&t->pmy, n) == cudaSuccess &&
              dev_alloc(&t->pmz, n) == cudaSuccess &&
              dev_alloc(&t->sort_hist, 2 * 256 * tiles) == cudaSuccess &&
              dev_alloc(&t->bt_count, kMaxLevel * (kBuildWarps + 1) * (tiles + 1) + 32) == cudaSuccess &&
              dev_alloc(&t->coh_bkt, n) == cudaSuccess && dev_alloc(&t->coh_cnt, 3 * ((n + kCohT - 1) / kCohT + 1) + 8) == cudaSuccess;
    t->cap_coh = ok ? 3 * ((n + kCohT - 1) / kCohT + 1) + 8 : 0;
    if (!ok) {
        cudaGetLastError();
        free_particles(t);
        return set_error(t->ctx, FDPS_ENOMEM, "device allocation for %lld particles failed",
                         (long long)n);
    }
    t->cap_n = n;
    t->cap_tiles = tiles;
    return FDPS_OK;
}

void free_nodes(fdps_tree* t) {
    dev_free(t->nd_first);
    dev_free(t->nd_count);
    dev_free(t->nd_child);
    dev_free(t->nd_meta);
    dev_free(t->nd_parent);
    dev_free(t->nd_qlo);
    dev_free(t->nd_sx);
    dev_free(t->nd_sy);
    dev_free(t->nd_sz);
    dev_free(t->nd_com);
    dev_free(t->nd_quad);
    dev_free(t->nd_f);
    dev_free(t->nd_walk);
    dev_free(t->nd_fq0);
    dev_free(t->nd_fq1);
    t->cap_nodes = 0;
}

int ensure_nodes(fdps_tree* t, int64_t cap) {
    if (cap <= t->cap_nodes) return FDPS_OK;
    free_nodes(t);
    bool ok = dev_alloc(&t->nd_first, cap) == cudaSuccess && dev_alloc(&t->nd_count, cap) == cudaSuccess &&
              dev_alloc(&t->nd_child, cap) == cudaSuccess && dev_alloc(&t->nd_meta, cap) == cudaSuccess &&
              dev_alloc(&t->nd_parent, cap) == cudaSuccess &&
              dev_alloc(&t->nd_qlo, cap) == cudaSuccess &&
              dev_alloc(&t->nd_sx, cap) == cudaSuccess &&
              dev_alloc(&t->nd_sy, cap) == cudaSuccess && dev_alloc(&t->nd_sz, cap) == cudaSuccess &&
              dev_alloc(&t->nd_com, cap) == cudaSuccess && dev_alloc(&t->nd_quad, 6 * cap) == cudaSuccess &&
              dev_alloc(&t->nd_f, 2 * cap) == cudaSuccess && dev_alloc(&t->nd_walk, cap) == cudaSuccess &&
              dev_alloc(&t->nd_fq0, cap) == cudaSuccess && dev_alloc(&t->nd_fq1, cap) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_nodes(t);
        return set_error(t->ctx, FDPS_ENOMEM, "device allocation for %lld nodes failed", (long long)cap);
    }
    t->cap_nodes = cap;
    return FDPS_OK;
}

void free_groups(fdps_tree* t) {
    dev_free(t->g_first);
    dev_free(t->g_count);
    dev_free(t->g_node);
    dev_free(t->g_box);
    dev_free(t->g_qbox);
    dev_free(t->g_ch);
    dev_free(t->g_cl);
    dev_free(t->g_blo);
    dev_free(t->g_bhi);
    dev_free(t->g_c64);
    dev_free(t->g_off);
    dev_free(t->g_len);
    dev_free(t->g_nspj);
    dev_free(t->g_nepj);
    t->cap_groups = 0;
}

int ensure_groups(fdps_tree* t, int64_t cap) {
    if (cap <= t->cap_groups) return FDPS_OK;
    free_groups(t);
    bool ok = dev_alloc(&t->g_first, cap) == cudaSuccess && dev_alloc(&t->g_count, cap) == cudaSuccess &&
              dev_alloc(&t->g_node, cap) == cudaSuccess && dev_alloc(&t->g_box, 6 * cap) == cudaSuccess &&
              dev_alloc(&t->g_qbox, 6 * cap) == cudaSuccess && dev_alloc(&t->g_ch, cap) == cudaSuccess &&
              dev_alloc(&t->g_cl, cap) == cudaSuccess && dev_alloc(&t->g_blo, cap) == cudaSuccess &&
              dev_alloc(&t->g_bhi, cap) == cudaSuccess && dev_alloc(&t->g_c64, cap) == cudaSuccess &&
              dev_alloc(&t->g_off, cap) == cudaSuccess && dev_alloc(&t->g_len, cap) == cudaSuccess &&
              dev_alloc(&t->g_nspj, cap) == cudaSuccess && dev_alloc(&t->g_nepj, cap) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_groups(t);
        return set_error(t->ctx, FDPS_ENOMEM, "device allocation for %lld groups failed", (long long)cap);
    }
    t->cap_groups = cap;
    return FDPS_OK;
}

int ensure_pool(fdps_tree* t, int64_t cap) {
    if (cap <= t->cap_pool) return FDPS_OK;
    dev_free(t->pool);
    t->cap_pool = 0;
    if (dev_alloc(&t->pool, cap) != cudaSuccess) {
        cudaGetLastError();
        return set_error(t->ctx, FDPS_ENOMEM, "device allocation of a %lld-entry list pool failed",
                         (long long)cap);
    }
    t->cap_pool = cap;
    return FDPS_OK;
}

int ensure_frontier(fdps_tree* t, int64_t per_warp) {
    if (per_warp <= t->cap_frontier) return FDPS_OK;
    dev_free(t->frontier);
    t->cap_frontier = 0;
    if (dev_alloc(&t->frontier, 2 * per_warp * t->n_walk_warps) != cudaSuccess) {
        cudaGetLastError();
        return set_error(t->ctx, FDPS_ENOMEM, "device allocation of walk frontiers failed");
    }
    t->cap_frontier = per_warp;
    return FDPS_OK;
}

int read_state(fdps_tree* t) {
    FDPS_CUDA_TRY(t->ctx, cudaMemcpyAsync(&t->h_st, t->st, sizeof(DevState), cudaMemcpyDeviceToHost,
                                          t->ctx->stream));
    FDPS_CUDA_TRY(t->ctx, cudaStreamSynchronize(t->ctx->stream));
    return FDPS_OK;
}

__global__ void k_reset_counters(DevState* st, int what) {
    if (threadIdx.x != 0) return;
    if (what & 1) {  // walk
        st->walk_counter = 0;
        st->pool_cursor = 0;
        st->pool_needed = 0;
        st->list_entries = 0;
        st->n_epj = 0;
        st->n_spj = 0;
        st->int_epj = 0;
        st->int_spj = 0;
        st->fallbacks = 0;
        st->max_frontier = 0;
        st->overflow &= ~(kOvfPool | kOvfChunk | kOvfFrontier);
    }
    if (what & 2) st->force_counter = 0;
    if (what & 4) {  // tree build
        st->overflow &= ~(kOvfNodes | kOvfGroups);
        st->mom_counter = 0;
        st->grp_done = 0;
    }
}

void record(fdps_tree* t, int k) {
    if (t->ev_ok && t->ctx->profiling && !t->ctx->capturing) cudaEventRecord(t->ev[k], t->ctx->stream);
}

int ensure_systems(fdps_tree* t, int64_t n_sys) {
    if (n_sys <= t->cap_sys) return FDPS_OK;
    dev_free(t->sys_box);
    t->cap_sys = 0;
    if (dev_alloc(&t->sys_box, n_sys) != cudaSuccess) {
        cudaGetLastError();
        return set_error(t->ctx, FDPS_ENOMEM, "device allocation for %lld system boxes failed",
                         (long long)n_sys);
    }
    t->cap_sys = n_sys;
    return FDPS_OK;
}

// The launches of one force calculation with the buffers as they are: no
// allocation, no host synchronisation (so it can be captured in a graph).
// Overflow of a buffer is left in the device state word.
int launch_force_pipeline(fdps_tree* t, fdps_psys* ps, int k_spj) {
    fdps_ctx* ctx = t->ctx;
    cudaStream_t s = ctx->stream;
    int rc;
    FDPS_CUDA_TRY(ctx, cudaMemsetAsync(t->st, 0, sizeof(DevState), s));
    if ((rc = keys_and_sort(t, ps))) return rc;
    if ((rc = reorder_particles(t, ps))) return rc;
    if ((rc = build_tree(t, ps))) return rc;
    if ((rc = compute_moments(t, ps))) return rc;
    if ((rc = select_groups(t, ps))) return rc;
    // the walk's and the force kernel's counters are still zero from the
    // state clear above (nothing between touches them): no reset launches
    if ((rc = launch_walk(t, ps->d_sys, (int)(t->n_walk_warps / walk_warps_per_block())))) return rc;
    return compute_forces(t, ps, k_spj);
}

int run_tree_stages(fdps_tree* t, fdps_psys* ps) {
    fdps_ctx* ctx = t->ctx;
    const int64_t n = ps->n;
    int rc;
    if (n >= (int64_t(1) << 30))
        return set_error(ctx, FDPS_EINVAL, "the tree handles fewer than 2^30 particles");
    if ((rc = ensure_particles(t, n))) return rc;
    if ((rc = ensure_systems(t, ps->n_sys))) return rc;
    const int64_t nl = t->p.n_leaf, ng = t->p.n_grp;
    if ((rc = ensure_nodes(t, std::min<int64_t>(8 * n / nl, 3 * n) + 1024 + ps->n_sys))) return rc;
    if ((rc = ensure_groups(t, std::min<int64_t>(n, 8 * n / ng + 1024)))) return rc;
    if ((rc = ensure_pool(t, 32 * n + t->n_walk_warps * (int64_t)walk_chunk()))) return rc;
    if ((rc = ensure_frontier(t, 4096))) return rc;
    t->n = n;
    t->valid = false;
    cudaStream_t s = ctx->stream;
    // a coherent sort whose bucket did not fit leaves the particles in
    // their order (the kernels after it copy them as they are): the call
    // starts over with the radix sort
    for (int sort_try = 0;; ++sort_try) {
    FDPS_CUDA_TRY(ctx, cudaMemsetAsync(t->st, 0, sizeof(DevState), s));
    record(t, 0);
    if ((rc = keys_and_sort(t, ps))) return rc;
    record(t, 2);
    if ((rc = reorder_particles(t, ps))) return rc;
    record(t, 3);
    bool redo = false;
    for (int attempt = 0;; ++attempt) {
        if ((rc = build_tree(t, ps))) return rc;
        record(t, 4);
        if ((rc = compute_moments(t, ps))) return rc;
        record(t, 5);
        if ((rc = select_groups(t, ps))) return rc;
        record(t, 6);
        if ((rc = read_state(t))) return rc;
        const uint32_t ov = t->h_st.overflow;
        if (ov & kSortStall) {
            t->coh_ok = false;
            return set_error(ctx, FDPS_ETIMEOUT, "a radix-sort look-back wait exceeded its bound");
        }
        if (ov & kSortRedo) {
            if (sort_try > 0) return set_error(ctx, FDPS_ECUDA, "coherent sort asked for a second redo");
            t->coh_ok = false;
            ++t->retries;
            redo = true;
            break;
        }
        if (!(ov & (kOvfNodes | kOvfGroups))) break;
        if (attempt > 8)
            return set_error(ctx, FDPS_EOVERFLOW, "tree build did not fit after %d resizes", attempt);
        ++t->retries;
        if (ov & kOvfNodes)
            if ((rc = ensure_nodes(t, 2 * t->cap_nodes))) return rc;
        if (ov & kOvfGroups)
            if ((rc = ensure_groups(t, std::min<int64_t>(n, 2 * t->cap_groups)))) return rc;
        k_reset_counters<<<1, 32, 0, s>>>(t->st, 4);
        FDPS_LAUNCH_CHECK(ctx);
    }
    if (!redo) break;
    }
    return FDPS_OK;
}

int run_force(fdps_tree* t, fdps_psys* ps, int k_spj, bool lists_only = false) {
    fdps_ctx* ctx = t->ctx;
    int rc;
    if ((rc = run_tree_stages(t, ps))) return rc;
    cudaStream_t s = ctx->stream;
    const int wblocks = (int)(t->n_walk_warps / walk_warps_per_block());
    for (int attempt = 0;; ++attempt) {
        k_reset_counters<<<1, 32, 0, s>>>(t->st, 1);
        FDPS_LAUNCH_CHECK(ctx);
        if ((rc = launch_walk(t, ps->d_sys, wblocks))) return rc;
        record(t, 7);
        if ((rc = read_state(t))) return rc;
        const uint32_t ov = t->h_st.overflow;
        if (!(ov & (kOvfPool | kOvfFrontier))) break;
        if (attempt > 8)
            return set_error(ctx, FDPS_EOVERFLOW, "interaction lists did not fit after %d resizes",
                             attempt);
        ++t->retries;
        if (ov & kOvfFrontier)
            if ((rc = ensure_frontier(t, 2 * t->cap_frontier))) return rc;
        if (ov & kOvfPool) {
            const int64_t need = (int64_t)(t->h_st.pool_needed * 3 / 2) +
                                 2 * t->n_walk_warps * (int64_t)walk_chunk();
            if ((rc = ensure_pool(t, std::max<int64_t>(need, 2 * t->cap_pool)))) return rc;
        }
    }
    if (lists_only) {  // S0-S7 only: the lists stay for user interaction kernels
        FDPS_CUDA_TRY(ctx, cudaGetLastError());
        t->valid = true;
        t->lists_of = ps;
        return FDPS_OK;
    }
    k_reset_counters<<<1, 32, 0, s>>>(t->st, 2);
    FDPS_LAUNCH_CHECK(ctx);
    if ((rc = compute_forces(t, ps, k_spj))) return rc;
    record(t, 8);
    FDPS_CUDA_TRY(ctx, cudaGetLastError());
    t->valid = true;
    t->lists_of = ps;
    ps->has_forces = true;
    return FDPS_OK;
}

bool valid_params(const fdps_tree_params* p) {
    return p && p->theta >= 0.0 && p->theta < 1e6 && p->theta == p->theta && p->n_leaf >= 1 &&
           p->n_leaf <= kMaxLeaf && p->n_grp >= p->n_leaf && p->n_grp <= kMaxGrp &&
           (p->moment == FDPS_MONOPOLE || p->moment == FDPS_QUADRUPOLE) &&
           (p->precision == FDPS_FP32REL || p->precision == FDPS_FP64) &&
           (p->tile_depth == 0 || p->tile_depth == 256 || p->tile_depth == 512) &&
           (p->block == 0 || p->block == 64 || p->block == 128 || p->block == 256) &&
           (p->i_per_thread == 0 || p->i_per_thread == 2 || p->i_per_thread == 4 || p->i_per_thread == 5) &&
           !(p->block == 256 && p->i_per_thread != 2);
}

}  // namespace

namespace fdps {
int run_tree(fdps_tree* t, fdps_psys* ps) { return run_tree_stages(t, ps); }
int read_device_state(fdps_tree* t) { return read_state(t); }
}  // namespace fdps

extern "C" {

int fdps_init(int device, fdps_ctx** out) {
    if (!out) return FDPS_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return FDPS_EINVAL;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return FDPS_ECUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return FDPS_EINVAL;
    fdps_ctx* ctx = new (std::nothrow) fdps_ctx();
    if (!ctx) return FDPS_ENOMEM;
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete ctx;
        return FDPS_ECUDA;
    }
    ctx->stream = ctx->own_stream;
    if (fdps::keys_sort_setup(ctx) != FDPS_OK) {
        cudaStreamDestroy(ctx->own_stream);
        delete ctx;
        return FDPS_ECUDA;
    }
    *out = ctx;
    return FDPS_OK;
}

int fdps_finalize(fdps_ctx* ctx) {
    if (!ctx) return FDPS_EINVAL;
    cudaSetDevice(ctx->device);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
    return FDPS_OK;
}

const char* fdps_last_error(const fdps_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

void* fdps_get_stream(const fdps_ctx* ctx) { return ctx ? (void*)ctx->stream : nullptr; }

int fdps_set_stream(fdps_ctx* ctx, void* stream) {
    if (!ctx) return FDPS_EINVAL;
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
    return FDPS_OK;
}

int64_t fdps_kernel_launches(const fdps_ctx* ctx) { return ctx ? ctx->launches : -1; }

int fdps_selftest_bounded_wait(fdps_ctx* ctx) {
    if (!ctx) return FDPS_EINVAL;
    cudaSetDevice(ctx->device);
    uint32_t flags = 0;
    int rc = selftest_lookback_timeout(ctx, &flags);
    if (rc) return rc;
    if (flags & kSortStall) return set_error(ctx, FDPS_ETIMEOUT, "bounded wait gave up as designed");
    return FDPS_OK;
}

int fdps_set_profiling(fdps_ctx* ctx, int on) {
    if (!ctx) return FDPS_EINVAL;
    ctx->profiling = on != 0;
    return FDPS_OK;
}

int fdps_psys_create(fdps_ctx* ctx, int64_t n, fdps_psys** out) {
    if (!ctx || !out) return FDPS_EINVAL;
    *out = nullptr;
    if (n < 1 || n > 0x7FFFFFFFLL) return set_error(ctx, FDPS_EINVAL, "particle count %lld out of range", (long long)n);
    cudaSetDevice(ctx->device);
    fdps_psys* ps = new (std::nothrow) fdps_psys();
    if (!ps) return FDPS_ENOMEM;
    ps->ctx = ctx;
    ps->n = n;
    ps->max_sys_n = n;
    bool ok = true;
    for (int b = 0; b < 2; ++b)
        ok = ok && dev_alloc(&ps->x[b], n) == cudaSuccess && dev_alloc(&ps->y[b], n) == cudaSuccess &&
             dev_alloc(&ps->z[b], n) == cudaSuccess && dev_alloc(&ps->vx[b], n) == cudaSuccess &&
             dev_alloc(&ps->vy[b], n) == cudaSuccess && dev_alloc(&ps->vz[b], n) == cudaSuccess &&
             dev_alloc(&ps->m[b], n) == cudaSuccess && dev_alloc(&ps->eps[b], n) == cudaSuccess &&
             dev_alloc(&ps->id[b], n) == cudaSuccess;
    ok = ok && dev_alloc(&ps->ax, n) == cudaSuccess && dev_alloc(&ps->ay, n) == cudaSuccess &&
         dev_alloc(&ps->az, n) == cudaSuccess && dev_alloc(&ps->pot, n) == cudaSuccess &&
         dev_alloc(&ps->d_flag, 1) == cudaSuccess &&
         dev_alloc(&ps->d_red, energy_scratch_doubles()) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        fdps_psys_destroy(ps);
        return set_error(ctx, FDPS_ENOMEM, "device allocation for %lld particles failed", (long long)n);
    }
    *out = ps;
    return FDPS_OK;
}

int fdps_psys_destroy(fdps_psys* ps) {
    if (!ps) return FDPS_EINVAL;
    cudaSetDevice(ps->ctx->device);
    for (int b = 0; b < 2; ++b) {
        dev_free(ps->x[b]);
        dev_free(ps->y[b]);
        dev_free(ps->z[b]);
        dev_free(ps->vx[b]);
        dev_free(ps->vy[b]);
        dev_free(ps->vz[b]);
        dev_free(ps->m[b]);
        dev_free(ps->eps[b]);
        dev_free(ps->id[b]);
    }
    dev_free(ps->ax);
    dev_free(ps->ay);
    dev_free(ps->az);
    dev_free(ps->pot);
    dev_free(ps->d_flag);
    dev_free(ps->d_red);
    dev_free(ps->stage);
    dev_free(ps->inv);
    dev_free(ps->rec);
    dev_free(ps->d_off);
    dev_free(ps->d_order);
    dev_free(ps->d_sys);
    dev_free(ps->d_sys_red);
    dev_free(ps->d_cbs);
    dev_free(ps->d_cbsys);
    dev_free(ps->d_csfb);
    delete ps;
    return FDPS_OK;
}

int64_t fdps_psys_size(const fdps_psys* ps) { return ps ? ps->n : -1; }

}  // extern "C"

namespace {

// The address under which the current device reads a caller's host
// pointer directly (page-locked or managed memory: on this part a kernel
// moves data over the CPU-GPU link as fast as a copy does), else null:
// such data is staged by copies instead.
const double* device_view(const double* p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost && a.devicePointer) return static_cast<const double*>(a.devicePointer);
    return nullptr;
}

}  // namespace

extern "C" {

int fdps_psys_set(fdps_psys* ps, const double* pos3n, const double* vel3n, const double* mass,
                  const double* eps, int on_device) {
    if (!ps) return FDPS_EINVAL;
    fdps_ctx* ctx = ps->ctx;
    if (!pos3n || !mass || !eps) return set_error(ctx, FDPS_EINVAL, "pos, mass and eps are required");
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    const int64_t n = ps->n;
    // new data for particles the system already holds keeps their order
    // (the last force calculation's), so that the next sort starts close to
    // sorted; the first data after creation, after set_systems or after a
    // rejected set take the caller's order
    const bool keep = ps->has_data;
    ps->has_data = false;
    ps->has_forces = false;
    uint32_t bad = 0;
    const double* vp = on_device ? nullptr : device_view(pos3n);
    const double* vv = on_device ? nullptr : device_view(vel3n);
    const double* vm = on_device ? nullptr : device_view(mass);
    const double* ve = on_device ? nullptr : device_view(eps);
    if (on_device) {
        int rc = launch_scatter_in(ps, pos3n, vel3n, mass, eps, keep, &bad);
        if (rc) return rc;
    } else if (vp && vm && ve && (!vel3n || vv)) {
        // the device reads the caller's buffers over the link
        int rc = launch_scatter_in(ps, vp, vel3n ? vv : nullptr, vm, ve, keep, &bad);
        if (rc) return rc;
    } else {
        // host data is staged in the psys's transfer buffer
        if (!ps->stage && dev_alloc(&ps->stage, 10 * n) != cudaSuccess) {
            cudaGetLastError();
            ps->stage = nullptr;
            return set_error(ctx, FDPS_ENOMEM, "staging allocation failed");
        }
        double* st_pos = ps->stage;
        double* st_vel = st_pos + 3 * n;
        double* st_m = st_pos + 6 * n;
        double* st_e = st_pos + 7 * n;
        cudaError_t e1 = cudaMemcpyAsync(st_pos, pos3n, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s);
        cudaError_t e2 = vel3n ? cudaMemcpyAsync(st_vel, vel3n, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s)
                               : cudaSuccess;
        cudaError_t e3 = cudaMemcpyAsync(st_m, mass, sizeof(double) * n, cudaMemcpyHostToDevice, s);
        cudaError_t e4 = cudaMemcpyAsync(st_e, eps, sizeof(double) * n, cudaMemcpyHostToDevice, s);
        int rc = FDPS_OK;
        if (e1 || e2 || e3 || e4)
            rc = set_error(ctx, FDPS_ECUDA, "host to device copy failed");
        else
            rc = launch_scatter_in(ps, st_pos, vel3n ? st_vel : nullptr, st_m, st_e, keep, &bad);
        cudaStreamSynchronize(s);
        if (rc) return rc;
    }
    if (bad)
        return set_error(ctx, FDPS_EINVAL, "invalid particle data:%s%s%s%s",
                         (bad & 1) ? " non-finite position" : "", (bad & 2) ? " non-finite velocity" : "",
                         (bad & 4) ? " negative or non-finite mass" : "",
                         (bad & 8) ? " non-positive or non-finite eps" : "");
    if (!keep) ps->gen++;  // the order changed: the last sorted keys no longer apply
    ps->has_data = true;
    return FDPS_OK;
}

int fdps_psys_get(const fdps_psys* ps, double* pos3n, double* vel3n, double* acc3n, double* pot,
                  int on_device) {
    if (!ps) return FDPS_EINVAL;
    fdps_ctx* ctx = ps->ctx;
    if (!ps->has_data) return set_error(ctx, FDPS_ESTATE, "particle data not set");
    if ((acc3n || pot) && !ps->has_forces)
        return set_error(ctx, FDPS_ESTATE, "no force calculation yet");
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    const int64_t n = ps->n;
    fdps_psys* pm = const_cast<fdps_psys*>(ps);
    if (on_device) {
        int rc = launch_gather_out(pm, pos3n, vel3n, acc3n, pot);
        if (rc) return rc;
        FDPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        return FDPS_OK;
    }
    // the device writes the caller's buffers over the link where it can
    double* vp = const_cast<double*>(device_view(pos3n));
    double* vv = const_cast<double*>(device_view(vel3n));
    double* va = const_cast<double*>(device_view(acc3n));
    double* vq = const_cast<double*>(device_view(pot));
    if ((!pos3n || vp) && (!vel3n || vv) && (!acc3n || va) && (!pot || vq)) {
        int rc = launch_gather_out(pm, vp, vv, va, vq);
        if (rc) return rc;
        FDPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        return FDPS_OK;
    }
    if (!pm->stage && dev_alloc(&pm->stage, 10 * n) != cudaSuccess) {
        cudaGetLastError();
        pm->stage = nullptr;
        return set_error(ctx, FDPS_ENOMEM, "staging allocation failed");
    }
    double* stage = pm->stage;
    int rc = launch_gather_out(pm, pos3n ? stage : nullptr, vel3n ? stage + 3 * n : nullptr,
                               acc3n ? stage + 6 * n : nullptr, pot ? stage + 9 * n : nullptr);
    cudaError_t e = cudaSuccess;
    if (!rc) {
        if (pos3n && !e) e = cudaMemcpyAsync(pos3n, stage, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s);
        if (vel3n && !e) e = cudaMemcpyAsync(vel3n, stage + 3 * n, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s);
        if (acc3n && !e) e = cudaMemcpyAsync(acc3n, stage + 6 * n, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s);
        if (pot && !e) e = cudaMemcpyAsync(pot, stage + 9 * n, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
        cudaError_t e2 = cudaStreamSynchronize(s);
        if (!e) e = e2;
    }
    if (rc) return rc;
    if (e) return set_error(ctx, FDPS_ECUDA, "device to host copy failed: %s", cudaGetErrorString(e));
    return FDPS_OK;
}

int fdps_tree_create(fdps_ctx* ctx, const fdps_tree_params* params, fdps_tree** out) {
    if (!ctx || !out) return FDPS_EINVAL;
    *out = nullptr;
    if (!valid_params(params))
        return set_error(ctx, FDPS_EINVAL,
                         "invalid tree parameters (theta >= 0, 1 <= n_leaf <= %d, n_leaf <= n_grp <= %d, "
                         "tile_depth 0/256/512, block 0/64/128/256, i_per_thread 0/2/4/5, block 256 with "
                         "i_per_thread 2)",
                         kMaxLeaf, kMaxGrp);
    cudaSetDevice(ctx->device);
    fdps_tree* t = new (std::nothrow) fdps_tree();
    if (!t) return FDPS_ENOMEM;
    t->ctx = ctx;
    t->p = *params;
    t->box_blocks = std::min(1024, ctx->sm_count * 4);
    t->n_walk_warps = (int64_t)walk_blocks(ctx) * walk_warps_per_block();
    bool ok = dev_alloc(&t->st, 1) == cudaSuccess && dev_alloc(&t->box_part, t->box_blocks) == cudaSuccess &&
              dev_alloc(&t->grp_scan, t->box_blocks) == cudaSuccess &&
              dev_alloc(&t->sort_dtot, 4096) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        fdps_tree_destroy(t);
        return set_error(ctx, FDPS_ENOMEM, "tree allocation failed");
    }
    t->ev_ok = true;
    for (int k = 0; k < 10; ++k)
        if (cudaEventCreate(&t->ev[k]) != cudaSuccess) t->ev_ok = false;
    cudaGetLastError();
    *out = t;
    return FDPS_OK;
}

int fdps_tree_destroy(fdps_tree* t) {
    if (!t) return FDPS_EINVAL;
    cudaSetDevice(t->ctx->device);
    free_particles(t);
    free_nodes(t);
    free_groups(t);
    dev_free(t->pool);
    dev_free(t->frontier);
    dev_free(t->st);
    dev_free(t->box_part);
    dev_free(t->grp_scan);
    dev_free(t->sort_dtot);
    dev_free(t->sys_box);
    dev_free(t->sr_h);
    dev_free(t->nd_hmax);
    dev_free(t->g_hmax);
    for (int k = 0; k < 10; ++k)
        if (t->ev[k]) cudaEventDestroy(t->ev[k]);
    delete t;
    return FDPS_OK;
}

int fdps_tree_calc_force_all_and_write_back(fdps_tree* t, fdps_psys* ps, int k_epj, int k_spj) {
    if (!t || !ps) return FDPS_EINVAL;
    fdps_ctx* ctx = t->ctx;
    if (ps->ctx != ctx) return set_error(ctx, FDPS_EINVAL, "tree and particle system belong to different contexts");
    if (k_epj != FDPS_GRAV_EPJ) return set_error(ctx, FDPS_EINVAL, "unknown EPJ kernel id %d", k_epj);
    if (k_spj != FDPS_GRAV_SPJ_MONO && k_spj != FDPS_GRAV_SPJ_QUAD)
        return set_error(ctx, FDPS_EINVAL, "unknown SPJ kernel id %d", k_spj);
    if (k_spj == FDPS_GRAV_SPJ_QUAD && t->p.moment != FDPS_QUADRUPOLE)
        return set_error(ctx, FDPS_EINVAL, "quadrupole SPJ kernel needs a quadrupole tree");
    if (!ps->has_data) return set_error(ctx, FDPS_ESTATE, "particle data not set");
    cudaSetDevice(ctx->device);
    return run_force(t, ps, k_spj);
}

int fdps_direct_sample(fdps_psys* ps, int64_t n_sample, const int64_t* rows, double* acc3, double* pot) {
    if (!ps || n_sample < 1 || !rows || (!acc3 && !pot)) return FDPS_EINVAL;
    fdps_ctx* ctx = ps->ctx;
    if (!ps->has_data) return set_error(ctx, FDPS_ESTATE, "particle data not set");
    for (int64_t k = 0; k < n_sample; ++k)
        if (rows[k] < 0 || rows[k] >= ps->n) return set_error(ctx, FDPS_EINVAL, "row %lld out of range", (long long)rows[k]);
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    int64_t* d_rows = nullptr;
    double* d_out = nullptr;
    if (cudaMalloc(&d_rows, sizeof(int64_t) * n_sample) != cudaSuccess ||
        cudaMalloc(&d_out, sizeof(double) * 4 * n_sample) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_rows);
        return set_error(ctx, FDPS_ENOMEM, "sample allocation failed");
    }
    std::vector<double> h(4 * (size_t)n_sample);
    int rc = cudaMemcpyAsync(d_rows, rows, sizeof(int64_t) * n_sample, cudaMemcpyHostToDevice, s) == cudaSuccess
                 ? direct_sample_device(ps, n_sample, d_rows, d_out)
                 : set_error(ctx, FDPS_ECUDA, "row copy failed");
    if (!rc && cudaMemcpy(h.data(), d_out, sizeof(double) * 4 * n_sample, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = set_error(ctx, FDPS_ECUDA, "result copy failed");
    cudaFree(d_rows);
    cudaFree(d_out);
    if (rc) return rc;
    for (int64_t k = 0; k < n_sample; ++k) {
        if (acc3)
            for (int a = 0; a < 3; ++a) acc3[3 * k + a] = h[4 * k + a];
        if (pot) pot[k] = h[4 * k + 3];
    }
    return FDPS_OK;
}

int fdps_tree_choose_theta(fdps_tree* t, fdps_psys* ps, double target, int64_t n_sample,
                           const double* candidates, int32_t n_candidates, double* theta_out,
                           double* median_out) {
    if (!t || !ps || !(target > 0.0) || n_sample < 1 || (candidates && n_candidates < 1)) return FDPS_EINVAL;
    fdps_ctx* ctx = t->ctx;
    if (ps->ctx != ctx) return set_error(ctx, FDPS_EINVAL, "tree and particle system belong to different contexts");
    if (!ps->has_data) return set_error(ctx, FDPS_ESTATE, "particle data not set");
    std::vector<double> cand;
    if (candidates) {
        cand.assign(candidates, candidates + n_candidates);
    } else {
        for (int k = 2; k <= 10; ++k) cand.push_back(0.1 * k);
    }
    for (double c : cand)
        if (!(c >= 0.0 && c < 1e6)) return set_error(ctx, FDPS_EINVAL, "candidate opening angle %g", c);
    std::sort(cand.begin(), cand.end());
    cudaSetDevice(ctx->device);
    const int64_t ns = std::min<int64_t>(n_sample, ps->n);
    std::vector<int64_t> rows(ns);
    for (int64_t k = 0; k < ns; ++k) rows[k] = (int64_t)(((__int128)k * ps->n) / ns);  // evenly spaced rows
    int64_t* d_rows = nullptr;
    double *d_ref = nullptr, *d_tree = nullptr;
    if (cudaMalloc(&d_rows, sizeof(int64_t) * ns) != cudaSuccess ||
        cudaMalloc(&d_ref, sizeof(double) * 4 * ns) != cudaSuccess ||
        cudaMalloc(&d_tree, sizeof(double) * 4 * ns) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_rows);
        cudaFree(d_ref);
        return set_error(ctx, FDPS_ENOMEM, "sample allocation failed");
    }
    const int k_spj = t->p.moment == FDPS_QUADRUPOLE ? FDPS_GRAV_SPJ_QUAD : FDPS_GRAV_SPJ_MONO;
    const double theta0 = t->p.theta;
    std::vector<double> ref(4 * ns), got(4 * ns), err(ns);
    int rc = cudaMemcpy(d_rows, rows.data(), sizeof(int64_t) * ns, cudaMemcpyHostToDevice) == cudaSuccess
                 ? direct_sample_device(ps, ns, d_rows, d_ref)
                 : set_error(ctx, FDPS_ECUDA, "row copy failed");
    if (!rc && cudaMemcpy(ref.data(), d_ref, sizeof(double) * 4 * ns, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = set_error(ctx, FDPS_ECUDA, "result copy failed");
    double best = cand.front(), best_med = -1.0;
    for (size_t q = 0; !rc && q < cand.size(); ++q) {
        t->p.theta = cand[q];
        if ((rc = run_force(t, ps, k_spj))) break;
        if ((rc = gather_rows_device(ps, ns, d_rows, d_tree))) break;
        if (cudaMemcpy(got.data(), d_tree, sizeof(double) * 4 * ns, cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = set_error(ctx, FDPS_ECUDA, "result copy failed");
            break;
        }
        for (int64_t k = 0; k < ns; ++k) {
            double dn = 0.0, rn = 0.0;
            for (int a = 0; a < 3; ++a) {
                const double d = got[4 * k + a] - ref[4 * k + a];
                dn += d * d;
                rn += ref[4 * k + a] * ref[4 * k + a];
            }
            err[k] = rn > 0.0 ? std::sqrt(dn / rn) : std::sqrt(dn);
        }
        std::nth_element(err.begin(), err.begin() + ns / 2, err.end());
        const double med = err[ns / 2];
        if (q == 0 || med <= target) {
            best = cand[q];
            best_med = med;
        }
        if (med > target) break;  // larger angles only lose accuracy
    }
    cudaFree(d_rows);
    cudaFree(d_ref);
    cudaFree(d_tree);
    if (rc) {
        t->p.theta = theta0;
        return rc;
    }
    t->p.theta = best;
    if ((rc = run_force(t, ps, k_spj))) return rc;  // leave the forces of the chosen angle
    if (theta_out) *theta_out = best;
    if (median_out) *median_out = best_med;
    return FDPS_OK;
}

int fdps_tree_neighbors(fdps_tree* t, fdps_psys* ps, int32_t mode, double r_fixed, const double* h,
                        int h_on_device, uint32_t* counts, double* rho, int out_on_device, int64_t* info3) {
    if (!t || !ps) return FDPS_EINVAL;
    fdps_ctx* ctx = t->ctx;
    if (ps->ctx != ctx) return set_error(ctx, FDPS_EINVAL, "tree and particle system belong to different contexts");
    if (mode < FDPS_CUTOFF_FIXED || mode > FDPS_CUTOFF_SYMMETRIC)
        return set_error(ctx, FDPS_EINVAL, "unknown cutoff type %d", (int)mode);
    if (mode == FDPS_CUTOFF_FIXED && !(r_fixed > 0.0 && r_fixed < 1e300))
        return set_error(ctx, FDPS_EINVAL, "the fixed cutoff needs a positive finite radius");
    if (mode != FDPS_CUTOFF_FIXED && !h) return set_error(ctx, FDPS_EINVAL, "this cutoff type needs radii");
    if (!ps->has_data) return set_error(ctx, FDPS_ESTATE, "particle data not set");
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    const int64_t n = ps->n;
    int rc;
    if ((rc = run_tree_stages(t, ps))) return rc;
    t->lists_of = nullptr;  // the pool will hold neighbour lists, not gravity lists
    double* d_h = nullptr;
    uint32_t* d_cnt = nullptr;
    double* d_rho = nullptr;
    unsigned long long* d_info = nullptr;
    auto cleanup = [&]() {
        if (d_h && !h_on_device) cudaFree(d_h);
        if (d_cnt && !out_on_device) cudaFree(d_cnt);
        if (d_rho && !out_on_device) cudaFree(d_rho);
        cudaFree(d_info);
    };
    if (mode != FDPS_CUTOFF_FIXED) {
        if (h_on_device) {
            d_h = const_cast<double*>(h);
        } else if (cudaMalloc(&d_h, sizeof(double) * n) != cudaSuccess ||
                   cudaMemcpyAsync(d_h, h, sizeof(double) * n, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            cleanup();
            return set_error(ctx, FDPS_ENOMEM, "radii transfer failed");
        }
    }
    if ((rc = short_prepare(t, ps, mode, d_h))) {
        cleanup();
        return rc;
    }
    const int wblocks = (int)(t->n_walk_warps / walk_warps_per_block());
    for (int attempt = 0;; ++attempt) {
        k_reset_counters<<<1, 32, 0, s>>>(t->st, 1);
        FDPS_LAUNCH_CHECK(ctx);
        if ((rc = launch_short_walk(t, ps, mode, r_fixed, wblocks)) || (rc = read_state(t))) {
            cleanup();
            return rc;
        }
        const uint32_t ov = t->h_st.overflow;
        if (!(ov & (kOvfPool | kOvfFrontier))) break;
        if (attempt > 8) {
            cleanup();
            return set_error(ctx, FDPS_EOVERFLOW, "neighbour lists did not fit after %d resizes", attempt);
        }
        ++t->retries;
        if ((ov & kOvfFrontier) && (rc = ensure_frontier(t, 2 * t->cap_frontier))) {
            cleanup();
            return rc;
        }
        if (ov & kOvfPool) {
            const int64_t need = (int64_t)(t->h_st.pool_needed * 3 / 2) +
                                 2 * t->n_walk_warps * (int64_t)walk_chunk();
            if ((rc = ensure_pool(t, std::max<int64_t>(need, 2 * t->cap_pool)))) {
                cleanup();
                return rc;
            }
        }
    }
    record(t, 7);  // stage times: ms_walk = radii preparation + walk, ms_force = pair pass
    if (out_on_device) {
        d_cnt = counts;
        d_rho = rho;
    }
    if ((!d_cnt && cudaMalloc(&d_cnt, sizeof(uint32_t) * n) != cudaSuccess) ||
        (!d_rho && cudaMalloc(&d_rho, sizeof(double) * n) != cudaSuccess) ||
        cudaMalloc(&d_info, sizeof(unsigned long long) * 3) != cudaSuccess ||
        cudaMemsetAsync(d_info, 0, sizeof(unsigned long long) * 3, s) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return set_error(ctx, FDPS_ENOMEM, "neighbour output allocation failed");
    }
    k_reset_counters<<<1, 32, 0, s>>>(t->st, 2);
    FDPS_LAUNCH_CHECK(ctx);
    if ((rc = launch_short_pairs(t, ps, mode, r_fixed, d_cnt, d_rho, d_info))) {
        cleanup();
        return rc;
    }
    record(t, 8);
    unsigned long long hinfo[3] = {0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(hinfo, d_info, sizeof(hinfo), cudaMemcpyDeviceToHost, s);
    if (!out_on_device) {
        if (!e && counts) e = cudaMemcpyAsync(counts, d_cnt, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, s);
        if (!e && rho) e = cudaMemcpyAsync(rho, d_rho, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    }
    const cudaError_t e2 = cudaStreamSynchronize(s);
    cleanup();
    if (e || e2) return set_error(ctx, FDPS_ECUDA, "neighbour results copy failed");
    if (info3)
        for (int k = 0; k < 3; ++k) info3[k] = (int64_t)hinfo[k];
    t->valid = true;
    return FDPS_OK;
}

int fdps_tree_build_lists(fdps_tree* t, fdps_psys* ps) {
    if (!t || !ps) return FDPS_EINVAL;
    fdps_ctx* ctx = t->ctx;
    if (ps->ctx != ctx) return set_error(ctx, FDPS_EINVAL, "tree and particle system belong to different contexts");
    if (!ps->has_data) return set_error(ctx, FDPS_ESTATE, "particle data not set");
    cudaSetDevice(ctx->device);
    const int k_spj = t->p.moment == FDPS_QUADRUPOLE ? FDPS_GRAV_SPJ_QUAD : FDPS_GRAV_SPJ_MONO;
    return run_force(t, ps, k_spj, true);
}

int fdps_tree_get_view(const fdps_tree* tc, const fdps_psys* ps, fdps_tree_view* v) {
    if (!tc || !ps || !v) return FDPS_EINVAL;
    fdps_tree* t = const_cast<fdps_tree*>(tc);
    if (!t->valid || t->lists_of != ps)
        return set_error(t->ctx, FDPS_ESTATE, "no lists of this particle system: build them first");
    if (t->p.precision != FDPS_FP32REL)
        return set_error(t->ctx, FDPS_EINVAL, "views are of FP32-relative trees");
    int rc = read_state(t);
    if (rc) return rc;
    *v = fdps_tree_view{};
    v->n = ps->n;
    v->n_groups = t->h_st.n_groups;
    v->quadrupole = t->p.moment == FDPS_QUADRUPOLE ? 1 : 0;
    v->leaf_tag = kLeafTag;
    v->g_first = t->g_first;
    v->g_count = t->g_count;
    v->g_off = t->g_off;
    v->g_len = t->g_len;
    v->g_ch = reinterpret_cast<const float*>(t->g_ch);
    v->g_cl = reinterpret_cast<const float*>(t->g_cl);
    v->pool = t->pool;
    v->nd_first = t->nd_first;
    v->nd_count = t->nd_count;
    v->nd_f = reinterpret_cast<const float*>(t->nd_f);
    v->nd_fq0 = v->quadrupole ? reinterpret_cast<const float*>(t->nd_fq0) : nullptr;
    v->nd_fq1 = v->quadrupole ? reinterpret_cast<const float*>(t->nd_fq1) : nullptr;
    v->pf_hi = reinterpret_cast<const float*>(t->pf_hi);
    v->pf_lo = reinterpret_cast<const float*>(t->pf_lo);
    v->id = ps->id[ps->cur];
    return FDPS_OK;
}

int fdps_kick(fdps_psys* ps, double dt_half) {
    if (!ps) return FDPS_EINVAL;
    if (!ps->has_forces) return set_error(ps->ctx, FDPS_ESTATE, "no force calculation yet");
    cudaSetDevice(ps->ctx->device);
    return launch_kick(ps, dt_half);
}

int fdps_drift(fdps_psys* ps, double dt) {
    if (!ps) return FDPS_EINVAL;
    if (!ps->has_data) return set_error(ps->ctx, FDPS_ESTATE, "particle data not set");
    cudaSetDevice(ps->ctx->device);
    return launch_drift(ps, dt);
}

int fdps_step(fdps_tree* t, fdps_psys* ps, double dt) {
    if (!t || !ps) return FDPS_EINVAL;
    if (!ps->has_forces) return set_error(ps->ctx, FDPS_ESTATE, "no force calculation yet");
    cudaSetDevice(ps->ctx->device);
    int rc;
    if ((rc = launch_kick_drift(ps, 0.5 * dt, dt))) return rc;
    const int k_spj = t->p.moment == FDPS_QUADRUPOLE ? FDPS_GRAV_SPJ_QUAD : FDPS_GRAV_SPJ_MONO;
    if ((rc = run_force(t, ps, k_spj))) return rc;
    return launch_kick(ps, 0.5 * dt);
}

int fdps_psys_energy(fdps_psys* ps, double* kinetic, double* potential) {
    if (!ps || !kinetic || !potential) return FDPS_EINVAL;
    if (!ps->has_forces) return set_error(ps->ctx, FDPS_ESTATE, "no force calculation yet");
    cudaSetDevice(ps->ctx->device);
    return launch_energy(ps, kinetic, potential);
}

int fdps_tree_get_stats(const fdps_tree* tc, fdps_tree_stats* out) {
    if (!tc || !out) return FDPS_EINVAL;
    fdps_tree* t = const_cast<fdps_tree*>(tc);
    if (!t->valid) return set_error(t->ctx, FDPS_ESTATE, "no force calculation yet");
    int rc = read_state(t);
    if (rc) return rc;
    memset(out, 0, sizeof(*out));
    const DevState& s = t->h_st;
    out->n_particles = t->n;
    out->n_nodes = s.n_nodes;
    out->n_groups = s.n_groups;
    out->n_levels = s.max_level + 1;
    out->list_entries = (int64_t)s.list_entries;
    out->n_epj = (int64_t)s.n_epj;
    out->n_spj = (int64_t)s.n_spj;
    out->interactions_epj = (int64_t)s.int_epj;
    out->interactions_spj = (int64_t)s.int_spj;
    out->fp64_fallbacks = (int64_t)s.fallbacks;
    out->retries = t->retries;
    out->sort_coherent = t->sort_coherent ? 1 : 0;
    if (t->ev_ok && t->ctx->profiling) {
        float v[9] = {0};
        for (int k = 0; k < 8; ++k)
            if (cudaEventElapsedTime(&v[k], t->ev[k], t->ev[k + 1]) != cudaSuccess) v[k] = -1.f;
        cudaGetLastError();
        float tot = 0.f;
        if (cudaEventElapsedTime(&tot, t->ev[0], t->ev[8]) != cudaSuccess) tot = -1.f;
        cudaGetLastError();
        out->ms_box_keys = v[0];
        out->ms_sort = v[1];
        out->ms_permute = v[2];
        out->ms_build = v[3];
        out->ms_moments = v[4];
        out->ms_groups = v[5];
        out->ms_walk = v[6];
        out->ms_force = v[7];
        out->ms_total = tot;
    }
    return FDPS_OK;
}

int fdps_tree_get_box(const fdps_tree* tc, double* out5) {
    if (!tc || !out5) return FDPS_EINVAL;
    fdps_tree* t = const_cast<fdps_tree*>(tc);
    if (!t->valid) return set_error(t->ctx, FDPS_ESTATE, "no force calculation yet");
    SysBox b;
    FDPS_CUDA_TRY(t->ctx, cudaMemcpyAsync(&b, t->sys_box, sizeof(SysBox), cudaMemcpyDeviceToHost,
                                          t->ctx->stream));
    FDPS_CUDA_TRY(t->ctx, cudaStreamSynchronize(t->ctx->stream));
    for (int a = 0; a < 3; ++a) out5[a] = b.lo[a];
    out5[3] = b.L;
    out5[4] = b.s;
    return FDPS_OK;
}

int fdps_tree_get_keys(const fdps_tree* tc, uint64_t* keys, uint32_t* perm, int64_t cap) {
    if (!tc) return FDPS_EINVAL;
    fdps_tree* t = const_cast<fdps_tree*>(tc);
    if (!t->valid) return set_error(t->ctx, FDPS_ESTATE, "no force calculation yet");
    if (cap < t->n) return set_error(t->ctx, FDPS_EOVERFLOW, "capacity %lld < %lld", (long long)cap, (long long)t->n);
    cudaStream_t s = t->ctx->stream;
    if (keys) FDPS_CUDA_TRY(t->ctx, cudaMemcpyAsync(keys, t->keys_in, 8 * t->n, cudaMemcpyDeviceToHost, s));
    if (perm) FDPS_CUDA_TRY(t->ctx, cudaMemcpyAsync(perm, t->perm, 4 * t->n, cudaMemcpyDeviceToHost, s));
    FDPS_CUDA_TRY(t->ctx, cudaStreamSynchronize(s));
    return FDPS_OK;
}

int fdps_tree_get_nodes(const fdps_tree* tc, int64_t cap, int64_t* n_out, int32_t* level, int64_t* first,
                        int64_t* count, int64_t* child_first, int32_t* nchild, double* mass, double* com,
                        double* quad) {
    if (!tc) return FDPS_EINVAL;
    fdps_tree* t = const_cast<fdps_tree*>(tc);
    if (!t->valid) return set_error(t->ctx, FDPS_ESTATE, "no force calculation yet");
    int rc = read_state(t);
    if (rc) return rc;
    const int64_t nn = t->h_st.n_nodes;
    if (n_out) *n_out = nn;
    if (cap < nn) return set_error(t->ctx, FDPS_EOVERFLOW, "capacity %lld < %lld nodes", (long long)cap, (long long)nn);
    cudaStream_t s = t->ctx->stream;
    uint32_t* h32 = (uint32_t*)malloc(4 * (size_t)nn * 4 + 1);
    double* h64 = (double*)malloc(sizeof(double) * (size_t)nn * 6 + 8);
    if (!h32 || !h64) {
        free(h32);
        free(h64);
        return set_error(t->ctx, FDPS_ENOMEM, "host allocation failed");
    }
    uint32_t *hf = h32, *hc = h32 + nn, *hch = h32 + 2 * nn, *hm = h32 + 3 * nn;
    cudaError_t e = cudaMemcpyAsync(hf, t->nd_first, 4 * nn, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(hc, t->nd_count, 4 * nn, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(hch, t->nd_child, 4 * nn, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(hm, t->nd_meta, 4 * nn, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (!e) {
        for (int64_t i = 0; i < nn; ++i) {
            const bool leaf = (hm[i] >> 16) & 1u;
            if (level) level[i] = (int32_t)(hm[i] & 0xFFu);
            if (first) first[i] = hf[i];
            if (count) count[i] = hc[i];
            if (child_first) child_first[i] = leaf ? -1 : (int64_t)hch[i];
            if (nchild) nchild[i] = leaf ? 0 : (int32_t)((hm[i] >> 8) & 0xFFu);
        }
        if (mass || com) {
            e = cudaMemcpyAsync(h64, t->nd_com, sizeof(dvec4) * nn, cudaMemcpyDeviceToHost, s);
            if (!e) e = cudaStreamSynchronize(s);
            for (int64_t i = 0; !e && i < nn; ++i) {
                if (mass) mass[i] = h64[4 * i + 3];
                if (com)
                    for (int a = 0; a < 3; ++a) com[3 * i + a] = h64[4 * i + a];
            }
        }
        if (quad && !e) {
            if (t->p.moment == FDPS_QUADRUPOLE && t->p.precision == FDPS_FP64) {
                e = cudaMemcpyAsync(quad, t->nd_quad, sizeof(double) * 6 * nn, cudaMemcpyDeviceToHost, s);
                if (!e) e = cudaStreamSynchronize(s);
            } else if (t->p.moment == FDPS_QUADRUPOLE) {
                // the FP32 pipeline keeps its quadrupoles in FP32
                float* hq = (float*)malloc(sizeof(float) * 6 * (size_t)nn + 8);
                if (!hq) e = cudaErrorMemoryAllocation;
                if (!e) e = cudaMemcpy2DAsync(hq, 6 * sizeof(float), t->nd_fq0, sizeof(float4), sizeof(float4),
                                              nn, cudaMemcpyDeviceToHost, s);
                if (!e) e = cudaMemcpy2DAsync(hq + 4, 6 * sizeof(float), t->nd_fq1, sizeof(float2),
                                              sizeof(float2), nn, cudaMemcpyDeviceToHost, s);
                if (!e) e = cudaStreamSynchronize(s);
                for (int64_t i = 0; !e && i < nn; ++i)
                    for (int k = 0; k < 6; ++k) quad[6 * i + k] = hq[6 * i + k];
                free(hq);
            } else {
                memset(quad, 0, sizeof(double) * 6 * nn);
            }
        }
    }
    free(h32);
    free(h64);
    if (e) return set_error(t->ctx, FDPS_ECUDA, "node readback failed: %s", cudaGetErrorString(e));
    return FDPS_OK;
}

int fdps_tree_get_groups(const fdps_tree* tc, int64_t cap, int64_t* n_out, int64_t* first, int64_t* count,
                         int64_t* node, double* box6) {
    if (!tc) return FDPS_EINVAL;
    fdps_tree* t = const_cast<fdps_tree*>(tc);
    if (!t->valid) return set_error(t->ctx, FDPS_ESTATE, "no force calculation yet");
    int rc = read_state(t);
    if (rc) return rc;
    const int64_t ng = t->h_st.n_groups;
    if (n_out) *n_out = ng;
    if (cap < ng) return set_error(t->ctx, FDPS_EOVERFLOW, "capacity %lld < %lld groups", (long long)cap, (long long)ng);
    cudaStream_t s = t->ctx->stream;
    uint32_t* h = (uint32_t*)malloc(4 * (size_t)ng * 3 + 4);
    if (!h) return set_error(t->ctx, FDPS_ENOMEM, "host allocation failed");
    cudaError_t e = cudaMemcpyAsync(h, t->g_first, 4 * ng, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(h + ng, t->g_count, 4 * ng, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(h + 2 * ng, t->g_node, 4 * ng, cudaMemcpyDeviceToHost, s);
    if (!e && box6) e = cudaMemcpyAsync(box6, t->g_box, sizeof(double) * 6 * ng, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (!e)
        for (int64_t g = 0; g < ng; ++g) {
            if (first) first[g] = h[g];
            if (count) count[g] = h[ng + g];
            if (node) node[g] = h[2 * ng + g];
        }
    free(h);
    if (e) return set_error(t->ctx, FDPS_ECUDA, "group readback failed: %s", cudaGetErrorString(e));
    return FDPS_OK;
}

int fdps_tree_get_lists(const fdps_tree* tc, int64_t g0, int64_t g1, int64_t* offsets, uint32_t* entries,
                        int64_t cap) {
    if (!tc || !offsets) return FDPS_EINVAL;
    fdps_tree* t = const_cast<fdps_tree*>(tc);
    if (!t->valid) return set_error(t->ctx, FDPS_ESTATE, "no force calculation yet");
    int rc = read_state(t);
    if (rc) return rc;
    const int64_t ng = t->h_st.n_groups;
    if (g0 < 0 || g1 < g0 || g1 > ng) return set_error(t->ctx, FDPS_EINVAL, "group range [%lld, %lld) out of [0, %lld)", (long long)g0, (long long)g1, (long long)ng);
    const int64_t m = g1 - g0;
    cudaStream_t s = t->ctx->stream;
    unsigned long long* hoff = (unsigned long long*)malloc(8 * (size_t)m + 8);
    uint32_t* hlen = (uint32_t*)malloc(4 * (size_t)m + 4);
    if (!hoff || !hlen) {
        free(hoff);
        free(hlen);
        return set_error(t->ctx, FDPS_ENOMEM, "host allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(hoff, t->g_off + g0, 8 * m, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(hlen, t->g_len + g0, 4 * m, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    int64_t tot = 0;
    offsets[0] = 0;
    for (int64_t k = 0; !e && k < m; ++k) {
        tot += hlen[k];
        offsets[k + 1] = tot;
    }
    if (!e && entries) {
        if (tot > cap) {
            free(hoff);
            free(hlen);
            return set_error(t->ctx, FDPS_EOVERFLOW, "capacity %lld < %lld entries", (long long)cap, (long long)tot);
        }
        for (int64_t k = 0; !e && k < m; ++k)
            if (hlen[k]) e = cudaMemcpyAsync(entries + offsets[k], t->pool + hoff[k], 4 * (size_t)hlen[k], cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
    }
    free(hoff);
    free(hlen);
    if (e) return set_error(t->ctx, FDPS_ECUDA, "list readback failed: %s", cudaGetErrorString(e));
    return FDPS_OK;
}

int fdps_tree_autotune(fdps_tree* t, fdps_psys* ps, const int32_t* n_leaf, int32_t n_nl,
                       const int32_t* n_grp, int32_t n_ng, const int32_t* tile_depth, int32_t n_td,
                       const int32_t* block, int32_t n_block, const int32_t* i_per_thread, int32_t n_ipt,
                       int32_t repeats, fdps_tree_params* best, double* best_ms) {
    if (!t || !ps || !n_leaf || !n_grp || n_nl < 1 || n_ng < 1 || repeats < 1) return FDPS_EINVAL;
    fdps_ctx* ctx = t->ctx;
    if (!ps->has_data) return set_error(ctx, FDPS_ESTATE, "particle data not set");
    cudaSetDevice(ctx->device);
    const int32_t td_default[1] = {0};
    if (!tile_depth || n_td < 1) {
        tile_depth = td_default;
        n_td = 1;
    }
    const int k_spj = t->p.moment == FDPS_QUADRUPOLE ? FDPS_GRAV_SPJ_QUAD : FDPS_GRAV_SPJ_MONO;
    cudaEvent_t e0, e1;
    FDPS_CUDA_TRY(ctx, cudaEventCreate(&e0));
    FDPS_CUDA_TRY(ctx, cudaEventCreate(&e1));
    const fdps_tree_params orig = t->p;
    fdps_tree_params win = orig;
    float win_ms = -1.f;
    int rc = FDPS_OK;
    // time one candidate: an untimed run (sizes the buffers) unless only the
    // force kernel's block shape changed, then the best of `repeats`
    auto trial = [&](const fdps_tree_params& cand, bool sizing) {
        t->p = cand;
        if (sizing && (rc = run_force(t, ps, k_spj))) return;
        float best_here = -1.f;
        for (int32_t r = 0; r < repeats && !rc; ++r) {
            cudaEventRecord(e0, ctx->stream);
            rc = run_force(t, ps, k_spj);
            cudaEventRecord(e1, ctx->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best_here < 0.f || ms < best_here) best_here = ms;
        }
        if (!rc && (win_ms < 0.f || best_here < win_ms)) {
            win_ms = best_here;
            win = cand;
        }
    };
    // stage 1: tree parameters at the tree's block shape
    for (int32_t a = 0; a < n_nl && !rc; ++a)
        for (int32_t b = 0; b < n_ng && !rc; ++b)
            for (int32_t c = 0; c < n_td && !rc; ++c) {
                fdps_tree_params cand = orig;
                cand.n_leaf = n_leaf[a];
                cand.n_grp = n_grp[b];
                cand.tile_depth = tile_depth[c];
                if (!valid_params(&cand)) continue;  // e.g. n_grp < n_leaf
                trial(cand, true);
            }
    // stage 2: the force kernel's block shape at stage 1's choice
    if (!rc && win_ms >= 0.f && t->p.precision == FDPS_FP32REL && ((block && n_block > 0) || (i_per_thread && n_ipt > 0))) {
        const fdps_tree_params base = win;
        const int32_t nb = (block && n_block > 0) ? n_block : 1;
        const int32_t ni = (i_per_thread && n_ipt > 0) ? n_ipt : 1;
        for (int32_t a = 0; a < nb && !rc; ++a)
            for (int32_t b = 0; b < ni && !rc; ++b) {
                fdps_tree_params cand = base;
                if (block && n_block > 0) cand.block = block[a];
                if (i_per_thread && n_ipt > 0) cand.i_per_thread = i_per_thread[b];
                if (!valid_params(&cand)) continue;  // e.g. block 256 with 4 i-particles
                if (cand.block == base.block && cand.i_per_thread == base.i_per_thread) continue;
                trial(cand, false);
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        t->p = orig;
        return rc;
    }
    if (win_ms < 0.f) {
        t->p = orig;
        return set_error(ctx, FDPS_EINVAL, "no valid candidate parameters");
    }
    t->p = win;
    if ((rc = run_force(t, ps, k_spj))) return rc;  // leave forces of the chosen parameters
    if (best) *best = win;
    if (best_ms) *best_ms = win_ms;
    return FDPS_OK;
}

int fdps_psys_set_systems(fdps_psys* ps, int32_t n_sys, const int64_t* offsets) {
    if (!ps) return FDPS_EINVAL;
    fdps_ctx* ctx = ps->ctx;
    if (n_sys < 1 || !offsets) return set_error(ctx, FDPS_EINVAL, "need n_sys >= 1 and offsets");
    if (offsets[0] != 0 || offsets[n_sys] != ps->n)
        return set_error(ctx, FDPS_EINVAL, "offsets must run from 0 to n = %lld", (long long)ps->n);
    for (int32_t k = 0; k < n_sys; ++k)
        if (offsets[k + 1] <= offsets[k])
            return set_error(ctx, FDPS_EINVAL, "system %d is empty or offsets decrease", (int)k);
    cudaSetDevice(ctx->device);
    dev_free(ps->d_off);
    dev_free(ps->d_order);
    dev_free(ps->d_sys);
    dev_free(ps->d_sys_red);
    dev_free(ps->d_cbs);
    dev_free(ps->d_cbsys);
    dev_free(ps->d_csfb);
    ps->coh_nb = 0;
    ps->n_sys = 1;
    ps->max_sys_n = ps->n;
    ps->gen++;
    ps->has_data = false;
    ps->has_forces = false;
    if (n_sys == 1) return FDPS_OK;
    if (dev_alloc(&ps->d_off, n_sys + 1) != cudaSuccess || dev_alloc(&ps->d_sys, ps->n) != cudaSuccess ||
        dev_alloc(&ps->d_sys_red, 2 * (int64_t)n_sys) != cudaSuccess ||
        dev_alloc(&ps->d_order, n_sys) != cudaSuccess) {
        cudaGetLastError();
        dev_free(ps->d_off);
        dev_free(ps->d_order);
        dev_free(ps->d_sys);
        dev_free(ps->d_sys_red);
        return set_error(ctx, FDPS_ENOMEM, "device allocation for %d systems failed", (int)n_sys);
    }
    ps->n_sys = n_sys;
    ps->max_sys_n = 0;
    for (int32_t k = 0; k < n_sys; ++k) ps->max_sys_n = std::max<int64_t>(ps->max_sys_n, offsets[k + 1] - offsets[k]);
    // per-system work (the moments) is handed out largest system first
    std::vector<int32_t> order(n_sys);
    for (int32_t k = 0; k < n_sys; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return offsets[a + 1] - offsets[a] > offsets[b + 1] - offsets[b];
    });
    FDPS_CUDA_TRY(ctx, cudaMemcpyAsync(ps->d_off, offsets, sizeof(int64_t) * (n_sys + 1),
                                       cudaMemcpyHostToDevice, ctx->stream));
    FDPS_CUDA_TRY(ctx, cudaMemcpyAsync(ps->d_order, order.data(), sizeof(int32_t) * n_sys,
                                       cudaMemcpyHostToDevice, ctx->stream));
    int rc = launch_sys_index(ps);
    if (rc) return rc;
    // buckets of the coherent time-step sort: each system's positions in
    // runs of kCohT (its last run ragged)
    std::vector<uint32_t> cbs, cbsys, csfb(n_sys + 1);
    for (int32_t k = 0; k < n_sys; ++k) {
        csfb[k] = (uint32_t)cbs.size();
        for (int64_t p = offsets[k]; p < offsets[k + 1]; p += kCohT) {
            cbs.push_back((uint32_t)p);
            cbsys.push_back((uint32_t)k);
        }
    }
    csfb[n_sys] = (uint32_t)cbs.size();
    const int64_t nbk = (int64_t)cbsys.size();
    cbs.push_back((uint32_t)ps->n);
    if (dev_alloc(&ps->d_cbs, nbk + 1) == cudaSuccess && dev_alloc(&ps->d_cbsys, nbk) == cudaSuccess &&
        dev_alloc(&ps->d_csfb, (int64_t)n_sys + 1) == cudaSuccess) {
        FDPS_CUDA_TRY(ctx, cudaMemcpyAsync(ps->d_cbs, cbs.data(), sizeof(uint32_t) * (nbk + 1),
                                           cudaMemcpyHostToDevice, ctx->stream));
        FDPS_CUDA_TRY(ctx, cudaMemcpyAsync(ps->d_cbsys, cbsys.data(), sizeof(uint32_t) * nbk,
                                           cudaMemcpyHostToDevice, ctx->stream));
        FDPS_CUDA_TRY(ctx, cudaMemcpyAsync(ps->d_csfb, csfb.data(), sizeof(uint32_t) * (n_sys + 1),
                                           cudaMemcpyHostToDevice, ctx->stream));
        ps->coh_nb = nbk;
    } else {
        // without the tables the ensemble keeps the radix sort
        cudaGetLastError();
        dev_free(ps->d_cbs);
        dev_free(ps->d_cbsys);
        dev_free(ps->d_csfb);
    }
    FDPS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return FDPS_OK;
}

int32_t fdps_psys_num_systems(const fdps_psys* ps) { return ps ? ps->n_sys : -1; }

int fdps_psys_energy_systems(fdps_psys* ps, double* kinetic, double* potential) {
    if (!ps || !kinetic || !potential) return FDPS_EINVAL;
    if (!ps->has_forces) return set_error(ps->ctx, FDPS_ESTATE, "no force calculation yet");
    cudaSetDevice(ps->ctx->device);
    return launch_energy_systems(ps, kinetic, potential);
}

int fdps_run(fdps_tree* t, fdps_psys* ps, double dt, int64_t n_steps) {
    if (!t || !ps) return FDPS_EINVAL;
    fdps_ctx* ctx = t->ctx;
    if (!ps->has_forces) return set_error(ctx, FDPS_ESTATE, "no force calculation yet");
    if (n_steps <= 0) return FDPS_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    const int k_spj = t->p.moment == FDPS_QUADRUPOLE ? FDPS_GRAV_SPJ_QUAD : FDPS_GRAV_SPJ_MONO;
    int rc = fdps_step(t, ps, dt);  // sizes every buffer
    if (rc || n_steps == 1) return rc;
    // headroom so that later steps rarely outgrow the captured buffers
    const DevState& h = t->h_st;
    if ((rc = ensure_nodes(t, h.n_nodes + h.n_nodes / 4 + 1024))) return rc;
    if ((rc = ensure_groups(t, std::min<int64_t>(ps->n, h.n_groups + h.n_groups / 4 + 1024)))) return rc;
    if ((rc = ensure_pool(t, (int64_t)(h.pool_needed * 3 / 2) + 2 * t->n_walk_warps * (int64_t)walk_chunk())))
        return rc;
    if ((rc = ensure_frontier(t, 2 * (int64_t)h.max_frontier + 1024))) return rc;
    const uint32_t ovf_mask = kOvfNodes | kOvfGroups | kOvfPool | kOvfFrontier | kSortStall | kSortRedo;
    // the particle buffers flip in every force calculation, so a step reads
    // buffer `cur` and leaves buffer 1 - cur: one graph for each parity
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    int64_t kernels[2] = {0, 0};  // kernel launches recorded in each graph
    for (int64_t k = 1; k < n_steps && !rc; ++k) {
        const int par = ps->cur;
        if (!exec[par]) {
            cudaGraph_t graph = nullptr;
            FDPS_CUDA_TRY(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            ctx->capturing = true;
            const int64_t l0 = ctx->launches;
            rc = launch_kick_drift(ps, 0.5 * dt, dt);
            if (!rc) rc = launch_force_pipeline(t, ps, k_spj);
            if (!rc) rc = launch_kick_guarded(ps, 0.5 * dt, &t->st->overflow, ovf_mask);
            ctx->capturing = false;
            kernels[par] = ctx->launches - l0;
            ctx->launches = l0;  // recorded, not launched; counted per replay
            ps->cur = par;  // capture only records; the flip happens on replay
            cudaError_t e = cudaStreamEndCapture(s, &graph);
            if (!rc && e != cudaSuccess)
                rc = set_error(ctx, FDPS_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
            if (!rc) {
                e = cudaGraphInstantiate(&exec[par], graph, 0);
                if (e != cudaSuccess)
                    rc = set_error(ctx, FDPS_ECUDA, "graph instantiation failed: %s",
                                   cudaGetErrorString(e));
            }
            if (graph) cudaGraphDestroy(graph);
            if (rc) break;
        }
        cudaError_t e = cudaGraphLaunch(exec[par], s);
        ctx->launches += kernels[par];
        uint32_t ov = 0;
        if (!e) e = cudaMemcpyAsync(&ov, &t->st->overflow, sizeof(ov), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) {
            rc = set_error(ctx, FDPS_ECUDA, "graph replay failed: %s", cudaGetErrorString(e));
            break;
        }
        ps->cur = 1 - par;  // the replayed reorder flipped the buffers
        if (ov & ovf_mask) {
            // this step's force overflowed: redo it with growing buffers (and
            // the radix sort), then the skipped kick; later steps recapture
            // with the new buffers
            ++t->retries;
            t->coh_ok = false;
            for (int q = 0; q < 2; ++q)
                if (exec[q]) {
                    cudaGraphExecDestroy(exec[q]);
                    exec[q] = nullptr;
                }
            if ((rc = run_force(t, ps, k_spj))) break;
            rc = launch_kick(ps, 0.5 * dt);
        }
    }
    for (int q = 0; q < 2; ++q)
        if (exec[q]) cudaGraphExecDestroy(exec[q]);
    if (rc) return rc;
    t->valid = true;
    ps->has_forces = true;
    return read_state(t);
}

}  // extern "C"
