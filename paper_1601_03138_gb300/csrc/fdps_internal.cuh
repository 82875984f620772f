// fdps_internal.cuh -- internal data layout of the CUDA Barnes-Hut library.
//
// Device memory is SoA.  Particles of a psys live in the order of the last
// force calculation (Morton order after the first call); `id` maps that
// order back to the caller's rows.  The tree keeps its own per-particle
// scratch (keys, sort buffers, FP32 hi/lo copies of the positions) and the
// node / group / list tables, all sized for the largest system seen and
// grown on demand.
#pragma once

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "../../include/fdps_gpu.h"

namespace fdps {

// Four doubles on a 32-byte boundary (one 256-bit load).
struct __align__(32) dvec4 {
    double x, y, z, w;
};
__host__ __device__ __forceinline__ dvec4 make_dvec4(double x, double y, double z, double w) {
    dvec4 v;
    v.x = x;
    v.y = y;
    v.z = z;
    v.w = w;
    return v;
}

constexpr int kMaxLevel = 21;           // 21 bits per axis, 63-bit keys
constexpr uint32_t kQMax = (1u << 21) - 1u;
constexpr uint32_t kLeafTag = 0x80000000u;  // list entry: opened leaf (EPJ)
constexpr int kMaxLeaf = 16;
constexpr int kMaxGrp = 4096;
constexpr int kBuildTile = 2048;  // positions per tile of the tree build
constexpr int kBuildWarps = 8;    // warps per tile of the tree build
constexpr int kCohT = 1024;       // positions per bucket of the coherent time-step sort

// overflow bits of DevState::overflow
constexpr uint32_t kOvfNodes = 1u;
constexpr uint32_t kOvfPool = 2u;
constexpr uint32_t kOvfFrontier = 4u;
constexpr uint32_t kOvfGroups = 8u;
constexpr uint32_t kBadInput = 16u;
constexpr uint32_t kOvfChunk = 32u;
constexpr uint32_t kSortStall = 64u;  // a radix-sort look-back wait gave up
constexpr uint32_t kSortRedo = 256u;  // a bucket of the coherent sort overflowed: redo with the radix sort
constexpr uint32_t kSortInvalid = kSortStall | kSortRedo;  // this call's order is not sorted
// Any of these leaves the step's lists or particle order invalid: the
// kernels downstream skip their work (the host redoes the step).
constexpr uint32_t kStepInvalid =
    kOvfNodes | kOvfPool | kOvfFrontier | kOvfGroups | kOvfChunk | kSortStall | kSortRedo;

// Per-tree device-resident state written by the kernels of one force call.
struct DevState {
    double lo[3];        // root box minimum
    double L;            // largest extent (1 if 0)
    double s;            // 2^21 / L
    double c0[3];        // root centre lo + L/2: origin of the FP32 hi/lo copies
    int32_t lvl_start[kMaxLevel + 3];  // node id range of each level
    int32_t n_nodes;
    int32_t n_groups;
    uint32_t overflow;
    uint32_t walk_counter;   // dynamic group scheduler of the walk
    uint32_t force_counter;  // dynamic group scheduler of the force kernel
    uint32_t mom_counter;    // dynamic system scheduler of the per-system moments
    uint32_t grp_done;       // blocks of the group count finished (the last one scans)
    uint32_t pad1;
    unsigned long long pool_cursor;  // list pool allocation cursor (entries)
    unsigned long long pool_needed;  // what the walk asked for, incl. overflow
    unsigned long long list_entries;
    unsigned long long n_epj;
    unsigned long long n_spj;
    unsigned long long int_epj;
    unsigned long long int_spj;
    unsigned long long fallbacks;
    uint32_t max_frontier;
    int32_t max_level;
};

// FP64 -> FP32 conversions on the integer pipes (GB300's FP64 pipe is
// narrow).  split_f32 gives hi = RN32(v) and lo = RN32(v - hi), the values
// of __double2float_rn(v) and __double2float_rn(v - (double)hi): the 53-bit
// significand rounded to nearest even at 24 bits, the remainder (exact in
// the 29 dropped bits, as an integer) converted by one correctly rounded
// int-to-float conversion and scaled by a power of two.  Values whose parts
// would leave the FP32 normal range take the FP64 instructions.
// The FP64 instructions for the rare values outside the integer path's
// exponent range, in a function of their own: inlined, the compiler may
// predicate them into the common path, where they would still take their
// cycles on the narrow FP64 pipe.
static __device__ __noinline__ float2 split_f32_fp64(double v) {
    const float hi = __double2float_rn(v);
    return make_float2(hi, __double2float_rn(v - (double)hi));
}
__device__ __forceinline__ void split_f32(double v, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e < 949 || e > 1149) {
        const float2 r = split_f32_fp64(v);
        hi = r.x;
        lo = r.y;
        return;
    }
    const unsigned long long sig = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    unsigned int keep = (unsigned int)(sig >> 29);
    const unsigned int rem = (unsigned int)(sig & 0x1FFFFFFFull);
    const bool up = rem > 0x10000000u || (rem == 0x10000000u && (keep & 1u));
    const int diff = (int)rem - (up ? 0x20000000 : 0);  // |v| - |hi| in units of 2^(e - 1075)
    keep += up ? 1u : 0u;
    int eh = e - 1023 + 127;
    if (keep == (1u << 24)) {  // rounded up to the next power of two
        keep >>= 1;
        ++eh;
    }
    const unsigned int sgn = (unsigned int)(b >> 63) << 31;
    hi = __uint_as_float(sgn | ((unsigned int)eh << 23) | (keep & 0x7FFFFFu));
    if (diff == 0) {
        lo = 0.0f;  // v - hi = +0
        return;
    }
    const float p2 = __uint_as_float((unsigned int)(e - 1075 + 127) << 23);
    lo = __uint_as_float(__float_as_uint(__fmul_rn(__int2float_rn(diff), p2)) ^ sgn);
}
// Grid coordinate of x (Sect. 3.2's key reading): q = min(2^21 - 1,
// floor((x - lo) s)) with the subtraction and the product rounded on their
// own.
__device__ __forceinline__ uint32_t quantise(double x, double lo, double s) {
    const double u = __dmul_rn(__dsub_rn(x, lo), s);
    // min(2^21 - 1, max(0, floor(u))) from the bits of u, on the integer
    // pipes (the FP64 pipe is narrow): u <= 0 or u < 1 give 0, u >= 2^21
    // the clamp, otherwise the significand shifted right by 52 - (e - 1023)
    const long long b = __double_as_longlong(u);
    if (b <= 0) return 0;  // +0, or negative (sign bit set)
    const int e = (int)(b >> 52);
    if (e < 1023) return 0;
    if (e >= 1023 + 21) return kQMax;
    const unsigned long long m = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    return (uint32_t)(m >> (52 - (e - 1023)));
}

__device__ __forceinline__ float to_f32(double v) {
    float hi, lo;
    split_f32(v, hi, lo);
    return hi;
}

// Root box of one system: lo = per-axis minimum, L = largest extent (1 if
// 0), s = 2^21 / L, c0 = lo + L/2 (origin of the FP32 hi/lo copies).
struct SysBox {
    double lo[3];
    double L;
    double s;
    double c0[3];
};

// Root-box reduction partials (one per block).
struct BoxPartial {
    double lo[3];
    double hi[3];
};

}  // namespace fdps

struct fdps_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    bool profiling = false;
    int64_t launches = 0;  // kernels launched by this library on this context
    bool capturing = false;  // a graph capture of a step is in progress
    std::string last_error;
};

struct fdps_psys {
    fdps_ctx* ctx = nullptr;
    int64_t n = 0;
    // current particle order (double-buffered for reordering)
    double* x[2] = {nullptr, nullptr};
    double* y[2] = {nullptr, nullptr};
    double* z[2] = {nullptr, nullptr};
    double* vx[2] = {nullptr, nullptr};
    double* vy[2] = {nullptr, nullptr};
    double* vz[2] = {nullptr, nullptr};
    double* m[2] = {nullptr, nullptr};
    double* eps[2] = {nullptr, nullptr};
    uint32_t* id[2] = {nullptr, nullptr};
    int cur = 0;
    // results of the last force calculation, in the current order
    double* ax = nullptr;
    double* ay = nullptr;
    double* az = nullptr;
    double* pot = nullptr;
    bool has_data = false;
    bool has_forces = false;
    uint64_t gen = 0;            // incremented whenever the particle data is replaced
    uint32_t* d_flag = nullptr;  // validation flag
    double* d_red = nullptr;     // reduction scratch (energy)
    double* stage = nullptr;     // host-transfer staging (10 n doubles, on first use)
    uint32_t* inv = nullptr;     // inverse of the current order (on first use)
    double* rec = nullptr;       // [n][8] records of new data in the current order (on first use)
    // independent systems: positions off[k] .. off[k+1] belong to system k;
    // with one system d_off and d_sys stay null
    int32_t n_sys = 1;
    int64_t max_sys_n = 0;       // particles of the largest system (n with one system)
    int64_t* d_off = nullptr;
    int32_t* d_order = nullptr;  // systems by decreasing particle count
    uint32_t* d_sys = nullptr;   // system of each position
    // buckets of the coherent time-step sort (several systems): bucket b
    // holds positions d_cbs[b] .. d_cbs[b + 1] - 1 of system d_cbsys[b];
    // system k's buckets start at d_csfb[k]
    uint32_t* d_cbs = nullptr;
    uint32_t* d_cbsys = nullptr;
    uint32_t* d_csfb = nullptr;
    int64_t coh_nb = 0;
    double* d_sys_red = nullptr; // per-system energies (2 n_sys)
};

struct fdps_tree {
    fdps_ctx* ctx = nullptr;
    fdps_tree_params p{};
    // per-particle scratch
    int64_t cap_n = 0;
    int64_t n = 0;  // particles of the last call
    uint64_t* keys_in = nullptr;   // keys in the call's starting order
    uint64_t* keys_a = nullptr;    // sort ping-pong
    uint64_t* keys_b = nullptr;
    uint32_t* vals_a = nullptr;
    uint32_t* vals_b = nullptr;
    uint32_t* perm = nullptr;      // result of the sort (points into vals_*)
    uint64_t* keys_sorted = nullptr;
    const fdps_psys* lists_of = nullptr;  // particle system of the current lists
    // short-range mode: cutoff radii in key order, per-node and per-group
    // maxima of the radii
    double* sr_h = nullptr;
    int64_t cap_sr_h = 0;
    double* nd_hmax = nullptr;
    int64_t cap_nd_hmax = 0;
    double* g_hmax = nullptr;
    int64_t cap_g_hmax = 0;
    // coherent sort: the sorted keys of the last call (keys_b) belong to
    // psys coh_ps at generation coh_gen, whose particles are in that order
    bool coh_ok = false;
    const fdps_psys* coh_ps = nullptr;
    uint64_t coh_gen = 0;
    int64_t coh_n = 0;
    bool sort_coherent = false;    // the last call took the coherent sort
    uint32_t* coh_bkt = nullptr;   // bucket of every particle
    uint32_t* coh_cnt = nullptr;   // [nb] counts, [nb + 1] offsets, [nb] cursors, done word
    int64_t cap_coh = 0;           // words of coh_cnt
    uint32_t* sort_hist = nullptr; // 2 x [tiles][256]: look-back words of the sort passes
    uint32_t* sort_dtot = nullptr; // [4096]: digit totals / bases of every pass, tile counters
    int64_t cap_tiles = 0;
    float4* pf_hi = nullptr;       // (x_hi, y_hi, z_hi, m) relative to c0
    float4* pf_lo = nullptr;       // (x_lo, y_lo, z_lo, eps^2)
    double* pmx = nullptr;         // m x, m y, m z of the sorted particles, each product rounded
    double* pmy = nullptr;         // once (the terms of the centre-of-mass sums, computed where
    double* pmz = nullptr;         // every lane has a particle)
    uint32_t* head = nullptr;      // per particle: group node starting here (tree build scratch before)
    uint32_t* bt_count = nullptr;  // tree build: per-warp node counts of each level, level totals
    // nodes
    int64_t cap_nodes = 0;
    uint32_t* nd_first = nullptr;
    uint32_t* nd_count = nullptr;
    uint32_t* nd_child = nullptr;   // first child id (0xFFFFFFFF for a leaf)
    uint32_t* nd_meta = nullptr;    // level | nchild << 8 | leaf << 16
    uint32_t* nd_parent = nullptr;
    uint64_t* nd_qlo = nullptr;     // packed grid origin x<<42 | y<<21 | z
    double* nd_sx = nullptr;        // FP64 sums of m x (bottom-up)
    double* nd_sy = nullptr;
    double* nd_sz = nullptr;
    fdps::dvec4* nd_com = nullptr;      // FP64 (com_x, com_y, com_z, M)
    double* nd_quad = nullptr;      // FP64 [n][6]
    float4* nd_f = nullptr;         // FP32 pairs [2i] = (com_hi - c0, M), [2i+1] = (com_lo, 0)
    uint4* nd_walk = nullptr;       // what one opening test reads: grid origin (2 words),
                                    // first child, meta
    float4* nd_fq0 = nullptr;       // FP32 (Qxx, Qyy, Qzz, Qxy)
    float2* nd_fq1 = nullptr;       // FP32 (Qxz, Qyz)
    // groups
    int64_t cap_groups = 0;
    uint32_t* g_first = nullptr;
    uint32_t* g_count = nullptr;
    uint32_t* g_node = nullptr;
    double* g_box = nullptr;        // FP64 [g][6] lo, hi
    uint32_t* g_qbox = nullptr;     // [g][6] qmin, qmax
    float4* g_ch = nullptr;         // FP32 (centre_hi - c0, 0)
    float4* g_cl = nullptr;         // FP32 (centre_lo, 0)
    float4* g_blo = nullptr;        // FP32 box minimum relative to centre
    float4* g_bhi = nullptr;        // FP32 box maximum relative to centre
    fdps::dvec4* g_c64 = nullptr;       // FP64 centre
    unsigned long long* g_off = nullptr;  // list offset in the pool
    uint32_t* g_len = nullptr;      // list length (entries)
    uint32_t* g_nspj = nullptr;     // SPJ entries
    uint32_t* g_nepj = nullptr;     // EPJ particles
    uint32_t* grp_scan = nullptr;   // compaction partials
    // lists
    int64_t cap_pool = 0;           // entries
    uint32_t* pool = nullptr;
    int64_t n_walk_warps = 0;
    int64_t cap_frontier = 0;       // entries per buffer per warp
    uint32_t* frontier = nullptr;
    // state
    fdps::DevState* st = nullptr;   // device
    fdps::DevState h_st{};          // host copy after a call
    fdps::BoxPartial* box_part = nullptr;
    int box_blocks = 0;
    fdps::SysBox* sys_box = nullptr;  // one per system
    int64_t cap_sys = 0;
    int64_t retries = 0;
    bool valid = false;
    // profiling
    cudaEvent_t ev[12] = {};
    bool ev_ok = false;
    float ms[10] = {};
};

namespace fdps {

// ---------------------------------------------------------------- errors

inline int set_error(fdps_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return code;
}

#define FDPS_CUDA_TRY(ctx, call)                                                  \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            return ::fdps::set_error((ctx), FDPS_ECUDA, "%s:%d %s: %s", __FILE__,  \
                                     __LINE__, #call, cudaGetErrorString(e_));    \
        }                                                                         \
    } while (0)

#define FDPS_LAUNCH_CHECK(ctx)                   \
    do {                                         \
        ++(ctx)->launches;                       \
        FDPS_CUDA_TRY(ctx, cudaGetLastError());  \
    } while (0)

template <class T>
inline cudaError_t dev_alloc(T** p, int64_t count) {
    *p = nullptr;
    if (count <= 0) count = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)count);
}

template <class T>
inline void dev_free(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

inline int grid_for(int64_t n, int block, int max_blocks) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

// --------------------------------------------------------- stage entry points
// (host functions, one per .cu file; all issue work on ctx->stream)

// S0-S6 of a force calculation (root box to i-groups, resizing on
// overflow) and a synchronous read of the device state word (api.cu)
int run_tree(fdps_tree* t, fdps_psys* ps);
int read_device_state(fdps_tree* t);
int keys_and_sort(fdps_tree* t, fdps_psys* ps);        // keys_sort.cu
int keys_sort_setup(fdps_ctx* ctx);                    // keys_sort.cu: once per context
int launch_sys_index(fdps_psys* ps);                   // integrate.cu
int launch_energy_systems(fdps_psys* ps, double* kin, double* pot);  // integrate.cu
int reorder_particles(fdps_tree* t, fdps_psys* ps);    // keys_sort.cu
int selftest_lookback_timeout(fdps_ctx* ctx, uint32_t* flags_out);  // keys_sort.cu
int build_tree(fdps_tree* t, fdps_psys* ps);           // build.cu
int compute_moments(fdps_tree* t, fdps_psys* ps);      // build.cu
int select_groups(fdps_tree* t, fdps_psys* ps);        // build.cu
int compute_forces(fdps_tree* t, fdps_psys* ps, int spj_kind);  // force.cu
// sampled rows (caller rows, device array): FP32-compensated direct sums
// and the last tree results, each as (ax, ay, az, phi) per row in d_out4
int direct_sample_device(fdps_psys* ps, int64_t ns, const int64_t* d_rows, double* d_out4);  // direct.cu
// short-range mode (short.cu): cutoff radii into key order (h_user: device,
// caller order) and their node and group maxima; the neighbour walk; the
// pair pass writing counts and densities in the caller's order.
int short_prepare(fdps_tree* t, fdps_psys* ps, int mode, const double* h_user);
int launch_short_walk(fdps_tree* t, fdps_psys* ps, int mode, double r_fixed, int blocks);
int launch_short_pairs(fdps_tree* t, fdps_psys* ps, int mode, double r_fixed, uint32_t* count,
                       double* rho, unsigned long long* info3);
int gather_rows_device(fdps_psys* ps, int64_t ns, const int64_t* d_rows, double* d_out4);    // direct.cu
int launch_kick(fdps_psys* ps, double dt_half);        // integrate.cu
int launch_kick_guarded(fdps_psys* ps, double dt_half, const uint32_t* flags, uint32_t mask);
int launch_drift(fdps_psys* ps, double dt);            // integrate.cu
int launch_kick_drift(fdps_psys* ps, double dt_half, double dt);  // integrate.cu
int launch_energy(fdps_psys* ps, double* kin, double* pot);  // integrate.cu
// caller-order input into the current buffers, validated (*bad: flag bits);
// keep_order: caller row i goes to the position the current order holds it
// at (id unchanged), else to position i (id = identity)
int launch_scatter_in(fdps_psys* ps, const double* pos, const double* vel,
                      const double* mass, const double* eps, bool keep_order, uint32_t* bad);  // integrate.cu
// current buffers and results out in the caller's order
int launch_gather_out(fdps_psys* ps, double* pos, double* vel,
                      double* acc, double* pot);       // integrate.cu

}  // namespace fdps
