// force.cu -- particle-particle (EPJ) and particle-superparticle (SPJ)
// forces from the interaction lists: one CTA per i-group (FP32-relative) or
// one warp per i-group (FP64 variant).
//
// Per i-particle (Sect. 2.2, Eqs. ParticleParticleNbody and
// ParticleSuperparticleNbody, G = 1, softening eps_i of the receiving
// particle):
//   a_i   = sum_EPJ m_j (x_j - x_i) / (r^2 + eps_i^2)^{3/2} + sum_SPJ f'
//   phi_i = -sum_EPJ m_j / (r^2 + eps_i^2)^{1/2} - ... + m_i / eps_i
// the last term removing the i-particle's own entry (its force term is zero).
// A quadrupole superparticle (mass M, traceless Q, r = x_i - com,
// R^2 = r^2 + eps_i^2) contributes phi = -M/R - (r.Q.r) / (2 R^5) and
// a = -M r / R^3 + Q r / R^5 - (5/2) (r.Q.r) r / R^7.  The FP32 kernel
// evaluates the same expressions regrouped as a = R^-5 (Q r + R^2 h r) and
// phi = R^-1 (h + 2 w), with w = (r.Q.r) R^-4 and h = -M - (5/2) w: 32 FP32
// operations per interaction (3 differences, 3 for R^2, 3 powers of 1/R,
// 9 for Q r, 3 for r.Q.r, w, h, R^2 h, 6 for a, 2 for phi) and one MUFU
// reciprocal square root.
//
// FP32-relative kernel (one CTA per i-group): list entries are gathered
// into shared memory as FP32 coordinates relative to the group centre,
// formed from FP32 hi/lo pairs so that near pairs keep full FP32 precision.
// A thread's i-particles are paired: the pair loop evaluates one list entry
// against two i-particles with packed two-lane FP32 instructions plus two
// MUFU rsqrt (one i-particle per thread: plain FP32); each thread
// accumulates one chunk of
// the list in plain FP32 and adds the chunk's sum to its running total with
// Kahan compensation.  Small groups split their list over several threads
// per i-particle ("slices"), reduced in FP64 at the end.  The FP64 kernel
// (one warp per group) is the same walk of the list on FP64 absolute
// coordinates with FP64 sums.
#include "fdps_internal.cuh"

namespace fdps {

struct ForceArgs {
    DevState* st;
    const uint32_t* g_first;
    const uint32_t* g_count;
    const unsigned long long* g_off;
    const uint32_t* g_len;
    const float4* g_ch;
    const float4* g_cl;
    const uint32_t* pool;
    const uint32_t* nd_first;
    const uint32_t* nd_count;
    const float4* nd_f;
    const float4* nd_fq0;
    const float2* nd_fq1;
    const dvec4* nd_com;
    const double* nd_quad;
    const float4* pf_hi;
    const float4* pf_lo;
    const double* px;
    const double* py;
    const double* pz;
    const double* pm;
    const double* peps;
    double* ax;
    double* ay;
    double* az;
    double* pot;
};

namespace {

constexpr int kFBlock = 128;
constexpr int kFWarps = kFBlock / 32;
constexpr int kJCap64 = 128;  // EPJ particles per FP64 tile

// Lane -> (i offset, slice) split of a group of n_i particles.
struct Split {
    int P, nsl;
    __device__ __forceinline__ Split(uint32_t ni) {
        if (ni <= 16u) {
            P = (int)ni;
            nsl = 32 / P;
        } else {
            P = 32;
            nsl = 1;
        }
    }
};

// Find the entry owning expanded item `item`: largest e with scan[e] <= item.
__device__ __forceinline__ int owner(const uint32_t* scan, uint32_t item) {
    int lo = 0, hi = 32;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (scan[mid] <= item)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- FP32
// One CTA of CB threads (64, 128 or 256: the "block shape" the autotuner
// picks, with the cap KMAX on i-particles per thread) per i-group.  Thread t
// owns K <= KMAX i-particles (i = t % P + k P, k < K) and the list slice
// j = t / P (mod nsl); (K, P, nsl) is chosen per group to keep the most
// lanes busy.  The list is consumed in chunks of 256 or 512 entries (the
// tile depth, EPT per thread); each chunk's superparticles and leaf
// particles are staged in shared memory, and each thread folds its FP32
// partial sums of the chunk into Kahan-compensated running sums once per
// chunk.

constexpr int kCJ = 224;  // leaf particles per shared tile (the shared memory of 128 x 5 fits 48 KB)

struct GroupPlan {
    int K, P, nsl;
};

template <int CB, int KMAX>
__device__ __forceinline__ GroupPlan plan_group(uint32_t ni) {
    // maximise ni * nsl / (CB * K) over K in {1, ..., 5} (up to KMAX);
    // larger K on ties
    GroupPlan best{1, 1, 1};
    float bu = -1.f;
    // an odd K is packed pairs plus one scalar lane: the scalar lane issues
    // as many instructions per list entry as a pair for half the work, so an
    // odd K must fill the CTA 6 % better to be taken
    constexpr float kOdd = 1.06f;
    const int Ks[5] = {5, 4, 3, 2, 1};
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const int K = Ks[c];
        if (K > KMAX) continue;
        const int P = (int)((ni + K - 1) / K);
        if (P > CB) continue;
        const int nsl = CB / P;
        const float u = (float)ni * nsl / (float)(CB * K) / ((K & 1) && K > 1 ? kOdd : 1.0f);
        if (u > bu + 1e-6f) {
            bu = u;
            best = GroupPlan{K, P, nsl};
        }
    }
    if (bu < 0.f) best = GroupPlan{KMAX, CB, 1};  // more than KMAX CB particles: rounds
    return best;
}

// Block-wide exclusive scans of two values at once (CB threads).
template <int CB>
__device__ __forceinline__ void block_scan2(uint32_t a, uint32_t b, uint32_t* ea, uint32_t* eb,
                                            uint32_t* ta, uint32_t* tb, uint32_t* s_w) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t va = __shfl_up_sync(0xFFFFFFFFu, ia, o);
        const uint32_t vb = __shfl_up_sync(0xFFFFFFFFu, ib, o);
        if (lane >= o) {
            ia += va;
            ib += vb;
        }
    }
    if (lane == 31) {
        s_w[w] = ia;
        s_w[CB / 32 + w] = ib;
    }
    __syncthreads();
    uint32_t oa = 0, ob = 0, sa = 0, sb = 0;
#pragma unroll
    for (int k = 0; k < CB / 32; ++k) {
        const uint32_t xa = s_w[k], xb = s_w[CB / 32 + k];
        if (k < w) {
            oa += xa;
            ob += xb;
        }
        sa += xa;
        sb += xb;
    }
    *ea = oa + ia - a;
    *eb = ob + ib - b;
    *ta = sa;
    *tb = sb;
}

// EPT consecutive u32 slots of one thread written as one vector.
template <int EPT>
__device__ __forceinline__ void store_entries(uint32_t* dst, const uint32_t (&v)[EPT]) {
    if (EPT == 8) {
        reinterpret_cast<uint4*>(dst)[0] = make_uint4(v[0], v[1 % EPT], v[2 % EPT], v[3 % EPT]);
        reinterpret_cast<uint4*>(dst)[1] = make_uint4(v[4 % EPT], v[5 % EPT], v[6 % EPT], v[7 % EPT]);
    } else if (EPT == 4)
        *reinterpret_cast<uint4*>(dst) = make_uint4(v[0], v[1 % EPT], v[2 % EPT], v[3 % EPT]);
    else if (EPT == 2)
        *reinterpret_cast<uint2*>(dst) = make_uint2(v[0], v[1 % EPT]);
    else
        for (int r = 0; r < EPT; ++r) dst[r] = v[r];
}

// Largest e in [0, CE) with scan[e] <= item (binary lifting: CE a power of
// two).
template <int CE>
__device__ __forceinline__ int owner_chunk(const uint32_t* scan, uint32_t item) {
    static_assert(CE > 0 && (CE & (CE - 1)) == 0, "list chunks of a power-of-two length");
    int lo = 0;
#pragma unroll
    for (int step = CE / 2; step > 0; step >>= 1)
        if (scan[lo + step] <= item) lo += step;
    return lo;
}

// hi + lo += v with an exact FP32 two-sum (Knuth): hi takes the rounded
// sum, lo the rounding error.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (v - bb);
    hi = s;
}

// Kahan running sums of one thread in shared memory: sum of (q, c) at
// s_k[((q * 4 + c) * 2) * CB + t], its compensation CB further on.
template <int CB>
__device__ __forceinline__ void kahan_smem_add(float* s_k, int q, int c, float v) {
    float* s = s_k + ((q * 4 + c) * 2) * CB + threadIdx.x;
    float* cp = s + CB;
    const float y = v - *cp;
    const float t = *s + y;
    *cp = (t - *s) - y;
    *s = t;
}

// Two FP32 lanes in one 64-bit register (low = i-particle 2h, high =
// 2h+1): each packed instruction evaluates one operation of the pair law
// for two interactions, halving the FP32 instructions the scheduler issues.
// Each lane is rounded exactly as the scalar instruction.
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_pk(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_up(f2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 f2_rsqrt(f2 v) {
    float a, b;
    f2_up(v, a, b);
    return f2_pk(rsqrtf(a), rsqrtf(b));
}
// Shared-memory layouts (coordinates relative to the group centre):
//   superparticles: float4 (x, y, z, -M), float4 (Qxx, Qyy, Qzz, Qxy),
//     float2 (Qxz, Qyz) in three arrays
//   leaf particles: float4 (x, y, z, m).
// A thread's i-particles are paired (2h, 2h+1) in the two lanes; each list
// entry is broadcast to both lanes.
template <bool QUAD>
struct SpjBuf {
    float4* s0;
    float4* s1;
    float2* s2;
};
__device__ __forceinline__ f2 f2_bc(float v) { return f2_pk(v, v); }

template <bool QUAD, int K, int EPT, int CB, int KMAX>
__device__ __forceinline__ void force_round_f32(const ForceArgs& A, uint32_t gf, uint32_t ni,
                                                unsigned long long off, uint32_t len, float4 gch,
                                                float4 gcl, int P, int nsl, uint32_t ib,
                                                float4* s_j, SpjBuf<QUAD> sb, uint32_t* s_ef,
                                                uint32_t* s_es, uint32_t* s_w,
                                                float* s_k) {
    constexpr int KP = K / 2;  // i-pairs; an odd K takes its last i-particle on the scalar path
    const int t = threadIdx.x;
    const int ip = t % P, sl = t / P;
    const bool on = sl < nsl;
    float xi[K], yi[K], zi[K], e2[K];
    bool iv[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        const uint32_t i = ib + (uint32_t)(ip + q * P);
        iv[q] = on && i < ni;
        xi[q] = yi[q] = zi[q] = 0.f;
        e2[q] = 1.f;
        if (iv[q]) {
            const float4 h = A.pf_hi[gf + i], l = A.pf_lo[gf + i];
            xi[q] = (h.x - gch.x) + (l.x - gcl.x);
            yi[q] = (h.y - gch.y) + (l.y - gcl.y);
            zi[q] = (h.z - gch.z) + (l.z - gcl.z);
            e2[q] = l.w;
        }
    }
    f2 xp[KP > 0 ? KP : 1], yp[KP > 0 ? KP : 1], zp[KP > 0 ? KP : 1], ep[KP > 0 ? KP : 1];
#pragma unroll
    for (int h = 0; h < KP; ++h) {
        xp[h] = f2_pk(xi[2 * h], xi[2 * h + 1]);
        yp[h] = f2_pk(yi[2 * h], yi[2 * h + 1]);
        zp[h] = f2_pk(zi[2 * h], zi[2 * h + 1]);
        ep[h] = f2_pk(e2[2 * h], e2[2 * h + 1]);
    }
    const f2 cm25 = f2_bc(-2.5f), c2 = f2_bc(2.0f);
    const int kbeg = on ? sl : 0x3FFFFFFF;
#pragma unroll
    for (int k = 0; k < 8 * K; ++k) s_k[k * CB + t] = 0.0f;

    constexpr int CE = CB * EPT;
    for (uint32_t base = 0; base < len; base += CE) {
        // ---- this thread's EPT consecutive entries: type, node data, leaf range
        uint32_t nspj = 0, npart = 0;
        uint32_t ent[EPT];
#pragma unroll
        for (int r = 0; r < EPT; ++r) {
            const uint32_t u = base + (uint32_t)(t * EPT + r);
            ent[r] = u < len ? A.pool[off + u] : 0xFFFFFFFFu;
        }
        uint32_t lcnt[EPT], lfirst[EPT];
#pragma unroll
        for (int r = 0; r < EPT; ++r) {
            const bool leaf = ent[r] != 0xFFFFFFFFu && (ent[r] & kLeafTag);
            const bool spj = ent[r] != 0xFFFFFFFFu && !(ent[r] & kLeafTag);
            lcnt[r] = leaf ? A.nd_count[ent[r] & ~kLeafTag] : 0u;
            lfirst[r] = leaf ? A.nd_first[ent[r] & ~kLeafTag] : 0u;
            nspj += spj ? 1u : 0u;
            npart += lcnt[r];
        }
        uint32_t rs, es, ns, total, esc[EPT];
        block_scan2<CB>(nspj, npart, &rs, &es, &ns, &total, s_w);
#pragma unroll
        for (int r = 0; r < EPT; ++r) {
            const bool spj = ent[r] != 0xFFFFFFFFu && !(ent[r] & kLeafTag);
            if (spj) {
                const uint32_t node = ent[r];
                const float4 fh = A.nd_f[2 * node], fl = A.nd_f[2 * node + 1];
                sb.s0[rs] = make_float4((fh.x - gch.x) + (fl.x - gcl.x),
                                        (fh.y - gch.y) + (fl.y - gcl.y),
                                        (fh.z - gch.z) + (fl.z - gcl.z), -fh.w);
                if (QUAD) {
                    sb.s1[rs] = A.nd_fq0[node];
                    sb.s2[rs] = A.nd_fq1[node];
                }
                ++rs;
            }
            esc[r] = es;
            es += lcnt[r];
        }
        // each thread's EPT consecutive slots in one vector store (no bank conflicts)
        store_entries<EPT>(s_ef + t * EPT, lfirst);
        store_entries<EPT>(s_es + t * EPT, esc);
        __syncthreads();
        float sax[K], say[K], saz[K], spp[K];  // scalar path (K = 1)
        f2 pax[KP > 0 ? KP : 1], pay[KP > 0 ? KP : 1], paz[KP > 0 ? KP : 1], pp[KP > 0 ? KP : 1];
#pragma unroll
        for (int q = 0; q < K; ++q) sax[q] = say[q] = saz[q] = spp[q] = 0.f;
#pragma unroll
        for (int h = 0; h < KP; ++h) pax[h] = pay[h] = paz[h] = pp[h] = 0ull;
        // ---- superparticles of this chunk
#pragma unroll 2
        for (int k = kbeg; k < (int)ns; k += nsl) {
            const float4 a = sb.s0[k];
            float4 q0;
            float2 q1;
            if (QUAD) {
                q0 = sb.s1[k];
                q1 = sb.s2[k];
            }
            if (K & 1) {  // the odd i-particle (index K - 1) in scalar FP32
                const float rx = xi[K - 1] - a.x, ry = yi[K - 1] - a.y, rz = zi[K - 1] - a.z;
                const float R2 = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, e2[K - 1])));
                const float Ri = rsqrtf(R2);
                const float Ri2 = Ri * Ri;
                if (QUAD) {
                    const float Ri4 = Ri2 * Ri2;
                    const float Ri5 = Ri4 * Ri;
                    const float Qrx = fmaf(q0.x, rx, fmaf(q0.w, ry, q1.x * rz));
                    const float Qry = fmaf(q0.w, rx, fmaf(q0.y, ry, q1.y * rz));
                    const float Qrz = fmaf(q1.x, rx, fmaf(q1.y, ry, q0.z * rz));
                    const float rQr = fmaf(rx, Qrx, fmaf(ry, Qry, rz * Qrz));
                    const float w = rQr * Ri4;                 // r.Q.r / R^4
                    const float hh = fmaf(-2.5f, w, a.w);      // -M - 5/2 w
                    const float hR2 = hh * R2;
                    sax[K - 1] = fmaf(Ri5, fmaf(hR2, rx, Qrx), sax[K - 1]);
                    say[K - 1] = fmaf(Ri5, fmaf(hR2, ry, Qry), say[K - 1]);
                    saz[K - 1] = fmaf(Ri5, fmaf(hR2, rz, Qrz), saz[K - 1]);
                    spp[K - 1] = fmaf(Ri, fmaf(2.0f, w, hh), spp[K - 1]);  // (-M - w/2) / R
                } else {
                    const float Ri3 = Ri * Ri2;
                    const float nMRi3 = a.w * Ri3;
                    sax[K - 1] = fmaf(nMRi3, rx, sax[K - 1]);
                    say[K - 1] = fmaf(nMRi3, ry, say[K - 1]);
                    saz[K - 1] = fmaf(nMRi3, rz, saz[K - 1]);
                    spp[K - 1] = fmaf(a.w, Ri, spp[K - 1]);
                }
            }
            if (KP > 0) {
                const f2 jx = f2_bc(a.x), jy = f2_bc(a.y), jz = f2_bc(a.z), nM = f2_bc(a.w);
                f2 qxx, qyy, qzz, qxy, qxz, qyz;
                if (QUAD) {
                    qxx = f2_bc(q0.x);
                    qyy = f2_bc(q0.y);
                    qzz = f2_bc(q0.z);
                    qxy = f2_bc(q0.w);
                    qxz = f2_bc(q1.x);
                    qyz = f2_bc(q1.y);
                }
#pragma unroll
                for (int h = 0; h < KP; ++h) {
                    const f2 rx = f2_sub(xp[h], jx), ry = f2_sub(yp[h], jy), rz = f2_sub(zp[h], jz);
                    const f2 R2 = f2_fma(rx, rx, f2_fma(ry, ry, f2_fma(rz, rz, ep[h])));
                    const f2 Ri = f2_rsqrt(R2);
                    const f2 Ri2 = f2_mul(Ri, Ri);
                    if (QUAD) {
                        const f2 Ri4 = f2_mul(Ri2, Ri2);
                        const f2 Ri5 = f2_mul(Ri4, Ri);
                        const f2 Qrx = f2_fma(qxx, rx, f2_fma(qxy, ry, f2_mul(qxz, rz)));
                        const f2 Qry = f2_fma(qxy, rx, f2_fma(qyy, ry, f2_mul(qyz, rz)));
                        const f2 Qrz = f2_fma(qxz, rx, f2_fma(qyz, ry, f2_mul(qzz, rz)));
                        const f2 rQr = f2_fma(rx, Qrx, f2_fma(ry, Qry, f2_mul(rz, Qrz)));
                        const f2 w = f2_mul(rQr, Ri4);         // r.Q.r / R^4
                        const f2 hh = f2_fma(cm25, w, nM);     // -M - 5/2 w
                        const f2 hR2 = f2_mul(hh, R2);
                        pax[h] = f2_fma(Ri5, f2_fma(hR2, rx, Qrx), pax[h]);
                        pay[h] = f2_fma(Ri5, f2_fma(hR2, ry, Qry), pay[h]);
                        paz[h] = f2_fma(Ri5, f2_fma(hR2, rz, Qrz), paz[h]);
                        pp[h] = f2_fma(Ri, f2_fma(c2, w, hh), pp[h]);  // (-M - w/2) / R
                    } else {
                        const f2 Ri3 = f2_mul(Ri, Ri2);
                        const f2 nMRi3 = f2_mul(nM, Ri3);  // -M/R^3
                        pax[h] = f2_fma(nMRi3, rx, pax[h]);
                        pay[h] = f2_fma(nMRi3, ry, pay[h]);
                        paz[h] = f2_fma(nMRi3, rz, paz[h]);
                        pp[h] = f2_fma(nM, Ri, pp[h]);
                    }
                }
            }
        }
        // ---- particles of the opened leaves, in shared tiles of kCJ
        for (uint32_t c0 = 0; c0 < total; c0 += kCJ) {
            const uint32_t m = total - c0 < (uint32_t)kCJ ? total - c0 : (uint32_t)kCJ;
            if (c0 > 0) __syncthreads();  // previous tile fully consumed
            for (uint32_t k = t; k < m; k += CB) {
                const uint32_t item = c0 + k;
                const int src = owner_chunk<CE>(s_es, item);
                const uint32_t p = s_ef[src] + (item - s_es[src]);
                const float4 h = A.pf_hi[p], l = A.pf_lo[p];
                s_j[k] = make_float4((h.x - gch.x) + (l.x - gcl.x), (h.y - gch.y) + (l.y - gcl.y),
                                     (h.z - gch.z) + (l.z - gcl.z), h.w);
            }
            __syncthreads();
#pragma unroll 2
            for (int k = kbeg; k < (int)m; k += nsl) {
                const float4 j = s_j[k];
                if (K & 1) {
                    const float dx = j.x - xi[K - 1], dy = j.y - yi[K - 1], dz = j.z - zi[K - 1];
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, e2[K - 1])));
                    const float ri = rsqrtf(r2);
                    const float mri = j.w * ri;
                    const float mri3 = mri * (ri * ri);
                    sax[K - 1] = fmaf(mri3, dx, sax[K - 1]);
                    say[K - 1] = fmaf(mri3, dy, say[K - 1]);
                    saz[K - 1] = fmaf(mri3, dz, saz[K - 1]);
                    spp[K - 1] -= mri;
                }
                if (KP > 0) {
                    const f2 jx = f2_bc(j.x), jy = f2_bc(j.y), jz = f2_bc(j.z), jm = f2_bc(j.w);
#pragma unroll
                    for (int h = 0; h < KP; ++h) {
                        const f2 dx = f2_sub(jx, xp[h]), dy = f2_sub(jy, yp[h]), dz = f2_sub(jz, zp[h]);
                        const f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_fma(dz, dz, ep[h])));
                        const f2 ri = f2_rsqrt(r2);
                        const f2 mri = f2_mul(jm, ri);
                        const f2 mri3 = f2_mul(mri, f2_mul(ri, ri));
                        pax[h] = f2_fma(mri3, dx, pax[h]);
                        pay[h] = f2_fma(mri3, dy, pay[h]);
                        paz[h] = f2_fma(mri3, dz, paz[h]);
                        pp[h] = f2_sub(pp[h], mri);
                    }
                }
            }
        }
        if (K & 1) {
            kahan_smem_add<CB>(s_k, K - 1, 0, sax[K - 1]);
            kahan_smem_add<CB>(s_k, K - 1, 1, say[K - 1]);
            kahan_smem_add<CB>(s_k, K - 1, 2, saz[K - 1]);
            kahan_smem_add<CB>(s_k, K - 1, 3, spp[K - 1]);
        }
#pragma unroll
        for (int h = 0; h < KP; ++h) {
            float lo, hi;
            f2_up(pax[h], lo, hi);
            kahan_smem_add<CB>(s_k, 2 * h, 0, lo);
            kahan_smem_add<CB>(s_k, 2 * h + 1, 0, hi);
            f2_up(pay[h], lo, hi);
            kahan_smem_add<CB>(s_k, 2 * h, 1, lo);
            kahan_smem_add<CB>(s_k, 2 * h + 1, 1, hi);
            f2_up(paz[h], lo, hi);
            kahan_smem_add<CB>(s_k, 2 * h, 2, lo);
            kahan_smem_add<CB>(s_k, 2 * h + 1, 2, hi);
            f2_up(pp[h], lo, hi);
            kahan_smem_add<CB>(s_k, 2 * h, 3, lo);
            kahan_smem_add<CB>(s_k, 2 * h + 1, 3, hi);
        }
        __syncthreads();  // chunk buffers are rewritten next
    }
    // ---- combine slices and write back.  A slice's Kahan pair (s, c) is the
    // double-float s + (-c); the combining thread of a row reads the pairs
    // of all its slices from the Kahan arrays, adds them with exact
    // two-sums in FP32 and turns each component into FP64 once (FP64 is a
    // narrow pipe on this part).  The potential's self term is removed with
    // the value the list's own entry contributed, m_i rsqrt(eps_i^2) in
    // FP32, so that the two cancel.
    const int rows = P * K;  // i-slots of this round: row r = ip + q P
    __syncthreads();         // every thread's Kahan sums are final
    for (int r = t; r < rows; r += CB) {
        const uint32_t i = ib + (uint32_t)r;
        if (i >= ni) continue;
        const int q = r / P, ipr = r - q * P;
        float hi[4] = {0.0f, 0.0f, 0.0f, 0.0f}, lo[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int s2 = 0; s2 < nsl; ++s2) {
            const int t2 = s2 * P + ipr;  // the thread of slice s2 holding row r
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                two_sum_acc(hi[c], lo[c], s_k[((q * 4 + c) * 2) * CB + t2]);
                lo[c] -= s_k[((q * 4 + c) * 2 + 1) * CB + t2];
            }
        }
        const uint32_t p = gf + i;
        two_sum_acc(hi[3], lo[3], A.pf_hi[p].w * rsqrtf(A.pf_lo[p].w));
        A.ax[p] = (double)hi[0] + (double)lo[0];
        A.ay[p] = (double)hi[1] + (double)lo[1];
        A.az[p] = (double)hi[2] + (double)lo[2];
        A.pot[p] = (double)hi[3] + (double)lo[3];
    }
    __syncthreads();
}

// Shared memory of the FP32 kernels (one CTA per group at a time).
template <bool QUAD, int EPT, int CB, int KMAX>
struct F32Shared {
    static constexpr int kCE = CB * EPT;
    static constexpr int kSpjBytes = kCE * (QUAD ? 40 : 16);
    __align__(16) unsigned char u[kSpjBytes];  // superparticles of a chunk
    __align__(16) float4 j[kCJ];
    __align__(16) uint32_t ef[kCE];
    __align__(16) uint32_t es[kCE];
    uint32_t w[2 * (CB / 32)];
    float k[KMAX * 8 * CB];  // Kahan sums and compensations
};

// Forces on the particles of group g, with the whole CTA.
template <bool QUAD, int EPT, int CB, int KMAX>
__device__ __forceinline__ void force_group(const ForceArgs& A, uint32_t g, F32Shared<QUAD, EPT, CB, KMAX>& sm) {
    constexpr int kCE = F32Shared<QUAD, EPT, CB, KMAX>::kCE;
    SpjBuf<QUAD> sb;
    sb.s0 = reinterpret_cast<float4*>(sm.u);
    sb.s1 = nullptr;  // a monopole chunk holds the first array only
    sb.s2 = nullptr;
    if constexpr (QUAD) {
        sb.s1 = reinterpret_cast<float4*>(sm.u + kCE * 16);
        sb.s2 = reinterpret_cast<float2*>(sm.u + kCE * 32);
    }
    const uint32_t ni = A.g_count[g], gf = A.g_first[g];
    const unsigned long long off = A.g_off[g];
    const uint32_t len = A.g_len[g];
    const float4 gch = A.g_ch[g], gcl = A.g_cl[g];
    for (uint32_t ib = 0; ib < ni;) {
        const GroupPlan pl = plan_group<CB, KMAX>(ni - ib);
        if (pl.K == 1) {
            force_round_f32<QUAD, 1, EPT, CB, KMAX>(A, gf, ni, off, len, gch, gcl, pl.P, pl.nsl, ib, sm.j, sb,
                                                    sm.ef, sm.es, sm.w, sm.k);
        } else if (KMAX >= 5 && pl.K == 5) {
            if constexpr (KMAX >= 5)
                force_round_f32<QUAD, 5, EPT, CB, KMAX>(A, gf, ni, off, len, gch, gcl, pl.P, pl.nsl, ib, sm.j, sb,
                                                        sm.ef, sm.es, sm.w, sm.k);
        } else if (KMAX >= 4 && pl.K == 3) {
            if constexpr (KMAX >= 4)
                force_round_f32<QUAD, 3, EPT, CB, KMAX>(A, gf, ni, off, len, gch, gcl, pl.P, pl.nsl, ib, sm.j, sb,
                                                        sm.ef, sm.es, sm.w, sm.k);
        } else if (KMAX == 2 || pl.K == 2) {
            force_round_f32<QUAD, 2, EPT, CB, KMAX>(A, gf, ni, off, len, gch, gcl, pl.P, pl.nsl, ib, sm.j, sb,
                                                    sm.ef, sm.es, sm.w, sm.k);
        } else {
            if constexpr (KMAX >= 4)
                force_round_f32<QUAD, 4, EPT, CB, KMAX>(A, gf, ni, off, len, gch, gcl, pl.P, pl.nsl, ib, sm.j,
                                                        sb, sm.ef, sm.es, sm.w, sm.k);
        }
        ib += (uint32_t)(pl.P * pl.K);
    }
}

// Up to 16 warps per SM (four 128-thread CTAs: 128 registers a thread).
template <bool QUAD, int EPT, int CB, int KMAX>
__global__ void __launch_bounds__(CB, (QUAD ? 512 / CB : 1)) k_force_f32(ForceArgs A) {
    __shared__ F32Shared<QUAD, EPT, CB, KMAX> sm;
    __shared__ uint32_t s_g;
    DevState* st = A.st;
    // lists cut short by a buffer overflow may point past the pool: no work
    // (a step replayed from a graph is redone by the host)
    if (st->overflow & kStepInvalid) return;
    const uint32_t ngroups = (uint32_t)st->n_groups;
    for (;;) {
        if (threadIdx.x == 0) s_g = atomicAdd(&st->force_counter, 1u);
        __syncthreads();
        const uint32_t g = s_g;
        __syncthreads();
        if (g >= ngroups) break;
        force_group<QUAD, EPT, CB, KMAX>(A, g, sm);
    }
}

template <bool QUAD>
__global__ void __launch_bounds__(kFBlock) k_force_f64(ForceArgs A) {
    __shared__ dvec4 s_j[kFWarps][kJCap64];
    __shared__ uint32_t s_ef[kFWarps][32];
    __shared__ uint32_t s_es[kFWarps][33];
    __shared__ double s_red[kFWarps][4][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    DevState* st = A.st;
    if (st->overflow & kStepInvalid) return;  // as in the FP32 kernel
    const uint32_t ngroups = (uint32_t)st->n_groups;
    for (;;) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(&st->force_counter, 1u);
        g = __shfl_sync(0xFFFFFFFFu, g, 0);
        if (g >= ngroups) break;
        const uint32_t ni = A.g_count[g], gf = A.g_first[g];
        const unsigned long long off = A.g_off[g];
        const uint32_t len = A.g_len[g];
        const Split sp(ni);
        const int ioff = lane % sp.P;
        const int sl = lane / sp.P;
        const bool lane_on = sl < sp.nsl;
        for (uint32_t ib = 0; ib < ni; ib += (uint32_t)sp.P) {
            const uint32_t i = ib + (uint32_t)ioff;
            const bool iv = lane_on && i < ni;
            double xi = 0.0, yi = 0.0, zi = 0.0, e2 = 1.0;
            if (iv) {
                xi = A.px[gf + i];
                yi = A.py[gf + i];
                zi = A.pz[gf + i];
                e2 = A.peps[gf + i] * A.peps[gf + i];
            }
            const int kbeg = iv ? sl : 0x7FFFFFFF;
            double ax = 0.0, ay = 0.0, az = 0.0, pp = 0.0;
            for (uint32_t t = 0; t < len; t += 32) {
                const bool ve = t + lane < len;
                const uint32_t e = ve ? A.pool[off + t + lane] : 0u;
                const bool isleaf = ve && (e & kLeafTag);
                const uint32_t node = e & ~kLeafTag;
                uint32_t cnt = 0, first = 0;
                if (isleaf) {
                    cnt = A.nd_count[node];
                    first = A.nd_first[node];
                }
                uint32_t inc = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                    if (lane >= o) inc += v;
                }
                const uint32_t total = __shfl_sync(0xFFFFFFFFu, inc, 31);
                s_ef[w][lane] = first;
                s_es[w][lane] = inc - cnt;
                // superparticles: every lane of a slice reads the entry from the pool
                const uint32_t nent = len - t < 32u ? len - t : 32u;
                for (int k = kbeg; k < (int)nent; k += sp.nsl) {
                    const uint32_t ek = A.pool[off + t + k];
                    if (ek & kLeafTag) continue;
                    const dvec4 c = A.nd_com[ek];
                    const double rx = xi - c.x, ry = yi - c.y, rz = zi - c.z;
                    const double R2 = rx * rx + ry * ry + rz * rz + e2;
                    const double Ri = rsqrt(R2);
                    const double Ri2 = Ri * Ri;
                    const double MRi = c.w * Ri;
                    const double MRi3 = MRi * Ri2;
                    ax -= MRi3 * rx;
                    ay -= MRi3 * ry;
                    az -= MRi3 * rz;
                    pp -= MRi;
                    if (QUAD) {
                        const double* Q = A.nd_quad + 6 * (int64_t)ek;
                        const double Qrx = Q[0] * rx + Q[3] * ry + Q[4] * rz;
                        const double Qry = Q[3] * rx + Q[1] * ry + Q[5] * rz;
                        const double Qrz = Q[4] * rx + Q[5] * ry + Q[2] * rz;
                        const double rQr = rx * Qrx + ry * Qry + rz * Qrz;
                        const double Ri5 = Ri2 * Ri2 * Ri;
                        const double c7 = 2.5 * rQr * Ri5 * Ri2;
                        ax += Qrx * Ri5 - c7 * rx;
                        ay += Qry * Ri5 - c7 * ry;
                        az += Qrz * Ri5 - c7 * rz;
                        pp -= 0.5 * rQr * Ri5;
                    }
                }
                __syncwarp();
                for (uint32_t c0 = 0; c0 < total; c0 += kJCap64) {
                    const uint32_t m = total - c0 < (uint32_t)kJCap64 ? total - c0 : (uint32_t)kJCap64;
                    for (uint32_t k = lane; k < m; k += 32) {
                        const uint32_t item = c0 + k;
                        const int src = owner(s_es[w], item);
                        const uint32_t p = s_ef[w][src] + (item - s_es[w][src]);
                        s_j[w][k] = make_dvec4(A.px[p], A.py[p], A.pz[p], A.pm[p]);
                    }
                    __syncwarp();
                    for (int k = kbeg; k < (int)m; k += sp.nsl) {
                        const dvec4 j = s_j[w][k];
                        const double dx = j.x - xi, dy = j.y - yi, dz = j.z - zi;
                        const double r2 = dx * dx + dy * dy + dz * dz + e2;
                        const double ri = rsqrt(r2);
                        const double mri = j.w * ri;
                        const double mri3 = mri * ri * ri;
                        ax += mri3 * dx;
                        ay += mri3 * dy;
                        az += mri3 * dz;
                        pp -= mri;
                    }
                    __syncwarp();
                }
                __syncwarp();
            }
            s_red[w][0][lane] = iv ? ax : 0.0;
            s_red[w][1][lane] = iv ? ay : 0.0;
            s_red[w][2][lane] = iv ? az : 0.0;
            s_red[w][3][lane] = iv ? pp : 0.0;
            __syncwarp();
            if (iv && sl == 0) {
                double r[4] = {0.0, 0.0, 0.0, 0.0};
                for (int s2 = 0; s2 < sp.nsl; ++s2)
#pragma unroll
                    for (int k = 0; k < 4; ++k) r[k] += s_red[w][k][s2 * sp.P + ioff];
                const uint32_t p = gf + i;
                A.ax[p] = r[0];
                A.ay[p] = r[1];
                A.az[p] = r[2];
                A.pot[p] = r[3] + A.pm[p] / A.peps[p];
            }
            __syncwarp();
        }
    }
}

}  // namespace

// One resident wave of FP32 force CTAs of the given shape (chunk CE
// entries, CB threads, at most KMAX i-particles a thread).
template <bool QUAD, int CE, int CB, int KMAX>
void launch_f32(const ForceArgs& A, fdps_ctx* ctx, cudaStream_t s) {
    constexpr int EPT = CE / CB;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force_f32<QUAD, EPT, CB, KMAX>, CB, 0) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    k_force_f32<QUAD, EPT, CB, KMAX><<<per_sm * ctx->sm_count, CB, 0, s>>>(A);
}

template <bool QUAD, int CE>
void launch_f32_shape(const ForceArgs& A, fdps_ctx* ctx, cudaStream_t s, int cb, int kmax) {
    if (cb == 64) {
        if (kmax == 2)
            launch_f32<QUAD, CE, 64, 2>(A, ctx, s);
        else if (kmax == 4)
            launch_f32<QUAD, CE, 64, 4>(A, ctx, s);
        else
            launch_f32<QUAD, CE, 64, 5>(A, ctx, s);
    } else if (cb == 256) {
        launch_f32<QUAD, CE, 256, 2>(A, ctx, s);  // 256 x 4 does not fit static shared memory
    } else {
        if (kmax == 2)
            launch_f32<QUAD, CE, 128, 2>(A, ctx, s);
        else if (kmax == 4)
            launch_f32<QUAD, CE, 128, 4>(A, ctx, s);
        else
            launch_f32<QUAD, CE, 128, 5>(A, ctx, s);
    }
}

int force_blocks_f64(fdps_ctx* ctx, int quad) {
    int per_sm = 0;
    const cudaError_t e = quad ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force_f64<true>, kFBlock, 0)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force_f64<false>, kFBlock, 0);
    if (e != cudaSuccess || per_sm < 1) per_sm = 4;
    return per_sm * ctx->sm_count;
}

ForceArgs force_args(fdps_tree* t, fdps_psys* ps) {
    const int c = ps->cur;
    ForceArgs A;
    A.st = t->st;
    A.g_first = t->g_first;
    A.g_count = t->g_count;
    A.g_off = t->g_off;
    A.g_len = t->g_len;
    A.g_ch = t->g_ch;
    A.g_cl = t->g_cl;
    A.pool = t->pool;
    A.nd_first = t->nd_first;
    A.nd_count = t->nd_count;
    A.nd_f = t->nd_f;
    A.nd_fq0 = t->nd_fq0;
    A.nd_fq1 = t->nd_fq1;
    A.nd_com = t->nd_com;
    A.nd_quad = t->nd_quad;
    A.pf_hi = t->pf_hi;
    A.pf_lo = t->pf_lo;
    A.px = ps->x[c];
    A.py = ps->y[c];
    A.pz = ps->z[c];
    A.pm = ps->m[c];
    A.peps = ps->eps[c];
    A.ax = ps->ax;
    A.ay = ps->ay;
    A.az = ps->az;
    A.pot = ps->pot;
    return A;
}

int compute_forces(fdps_tree* t, fdps_psys* ps, int spj_kind) {
    fdps_ctx* ctx = t->ctx;
    const ForceArgs A = force_args(t, ps);
    const bool quad = spj_kind == FDPS_GRAV_SPJ_QUAD;
    cudaStream_t s = ctx->stream;
    if (t->p.precision == FDPS_FP64) {
        const int blocks = force_blocks_f64(ctx, quad);
        if (quad)
            k_force_f64<true><<<blocks, kFBlock, 0, s>>>(A);
        else
            k_force_f64<false><<<blocks, kFBlock, 0, s>>>(A);
    } else {
        // tile depth: list entries staged per chunk (0 = default 512); block
        // shape: threads per CTA (0 = 128) and i-particles per thread (0 = 5)
        const bool shallow = t->p.tile_depth == 256;
        const int cb = t->p.block ? t->p.block : 128;
        const int kmax = t->p.i_per_thread ? t->p.i_per_thread : 5;
        if (quad) {
            if (shallow)
                launch_f32_shape<true, 256>(A, ctx, s, cb, kmax);
            else
                launch_f32_shape<true, 512>(A, ctx, s, cb, kmax);
        } else {
            if (shallow)
                launch_f32_shape<false, 256>(A, ctx, s, cb, kmax);
            else
                launch_f32_shape<false, 512>(A, ctx, s, cb, kmax);
        }
    }
    FDPS_LAUNCH_CHECK(ctx);
    return FDPS_OK;
}

}  // namespace fdps
