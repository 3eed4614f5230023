// pairs.cuh — shared pieces of the pair passes (Sinkhorn, M-step, adjoint):
// the packed pair evaluation, the online log-sum-exp, the dustbin scalars and
// the persistent-CTA pipeline that streams one side of an angle block through
// shared memory with bulk copies.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace laue {

constexpr int kTPB = 256;     // widest CTA of the pair passes (one row/column pair per thread)
constexpr int kChunk = 128;   // staged pairs per chunk (256 spots)
constexpr int kGran = kConeGran;  // pairs per cone granule of the exact skipping
constexpr int kParts = kChunk / kGran;  // granules per staged chunk
constexpr int kGroup = 4;     // staged pairs per max-then-sum group
constexpr float kPadFar = 1.0e6f;

struct DustPtrs {
    float *F0, *F0n, *G0, *log2U, *log2O, *Fmax, *Gmax, *err;
};

__device__ __forceinline__ DustPtrs dust_ptrs(float* base, int T) {
    DustPtrs d;
    d.F0 = base;
    d.F0n = base + T;
    d.G0 = base + 2 * T;
    d.log2U = base + 3 * T;
    d.log2O = base + 4 * T;
    d.Fmax = base + 5 * T;  // per-angle max of F (row potentials)
    d.Gmax = base + 6 * T;  // per-angle max of G (column potentials)
    d.err = base + 7 * T;
    return d;
}

// Packed pair value base + K |(p - c)/|p - c| - r|^2 for two pairs at once;
// nc = -c, nr = -r.  13 packed instructions and 2 MUFU rsqrt.
__device__ __forceinline__ f2 pair_v2(f2 px, f2 py, f2 pz, f2 ncx, f2 ncy, f2 ncz, f2 nrx, f2 nry, f2 nrz,
                                      f2 K2, f2 base) {
    f2 dx = add2(px, ncx), dy = add2(py, ncy), dz = add2(pz, ncz);
    f2 q = mul2(dx, dx);
    q = fma2(dy, dy, q);
    q = fma2(dz, dz, q);
    f2 s = pk(rsq(lo(q)), rsq(hi(q)));
    f2 ex = fma2(dx, s, nrx), ey = fma2(dy, s, nry), ez = fma2(dz, s, nrz);
    f2 e2 = mul2(ex, ex);
    e2 = fma2(ey, ey, e2);
    e2 = fma2(ez, ez, e2);
    return fma2(e2, K2, base);
}

// Online base-2 log-sum-exp state of one row: running max m and two packed
// partial sums S (relative to m).
struct RowLse {
    float m;
    f2 S;
    f2 nm;  // {-m, -m}
    __device__ __forceinline__ void init(float v) {
        m = v;
        S = pk(1.0f, 0.0f);
        nm = dup(-v);
    }
    // fold 8 values (4 packed) in: one max / rescale, 8 MUFU ex2
    __device__ __forceinline__ void add4(const f2 (&v)[kGroup]) {
        float c1 = max3(lo(v[0]), hi(v[0]), lo(v[1]));
        float c2 = max3(hi(v[1]), lo(v[2]), hi(v[2]));
        float cm = max3(c1, c2, fmaxf(lo(v[3]), hi(v[3])));
        if (cm > m) {
            float sc = ex2(m - cm);
            S = mul2(S, dup(sc));
            m = cm;
            nm = dup(-cm);
        }
#pragma unroll
        for (int g = 0; g < kGroup; ++g) {
            f2 t = add2(v[g], nm);
            S = add2(S, pk(ex2(lo(t)), ex2(hi(t))));
        }
    }
    __device__ __forceinline__ void add1(f2 v) {
        float cm = fmaxf(lo(v), hi(v));
        if (cm > m) {
            float sc = ex2(m - cm);
            S = mul2(S, dup(sc));
            m = cm;
            nm = dup(-cm);
        }
        f2 t = add2(v, nm);
        S = add2(S, pk(ex2(lo(t)), ex2(hi(t))));
    }
    __device__ __forceinline__ float value() const { return m + lg2(lo(S) + hi(S)); }
};

// Angle block of element k of a list with offsets off[T+1] (binary search).
__device__ __forceinline__ int block_of(const int* __restrict__ off, int T, int k) {
    int lo_ = 0, hi_ = T;
    while (hi_ - lo_ > 1) {
        int mid = (lo_ + hi_) >> 1;
        if (off[mid] <= k) lo_ = mid;
        else hi_ = mid;
    }
    return lo_;
}

// ------------------------------------------------------ staged chunk pipeline
constexpr int kMaxList = 512;  // chunks of one angle block a tile can list for skipping

struct Stage {
    float4 s[4][2][kChunk];  // up to 4 arrays x 2 stages
    uint64_t bar[2];
    int tile;
    int last;
    float red_m[kTPB / 32], red_s[kTPB / 32];
    int wcnt[kTPB / 32];
    int list[kMaxList];      // chunks of the streamed side this tile needs
};

struct Srcs {
    const float4* p[4];
    int n;  // number of arrays (2 or 4)
};

// Thread 0 issues the bulk copies of chunk `ch` of every source array into
// stage ch & 1.
__device__ __forceinline__ void issue_chunk(Stage& S, int ch, const Srcs& src, int base, int n_total) {
    int st = ch & 1;
    int n = min(kChunk, n_total - ch * kChunk);
    uint32_t bytes = (uint32_t)n * 16u;
    mbar_expect_tx(&S.bar[st], bytes * (uint32_t)src.n);
    for (int k = 0; k < src.n; ++k) bulk_g2s(S.s[k][st], src.p[k] + base + ch * kChunk, bytes, &S.bar[st]);
}

__device__ __forceinline__ void block_lse(Stage& S, float& m, float& s) {
    warp_lse_reduce(m, s);
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        S.red_m[w] = m;
        S.red_s[w] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Lse2 L;
        L.m = kNegHuge;
        L.s = 0.0f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) L.merge(S.red_m[k], S.red_s[k]);
        m = L.m;
        s = L.s;
    }
    __syncthreads();
}

__device__ __forceinline__ float block_max(Stage& S, float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) S.red_m[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = S.red_m[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) r = fmaxf(r, S.red_m[k]);
    __syncthreads();
    return r;
}

// Streams n_total pairs of every source array (from pair index `base`) through
// shared memory; per chunk, prep(stage, count) runs on all threads, a barrier
// makes its writes visible, then body(stage, count, offset) runs.  Returns
// false (uniformly across the CTA) when a bounded wait ran out.
template <class Prep, class Body>
__device__ __forceinline__ bool stream_tile_prep(Stage& S, uint32_t (&parity)[2], const Srcs& src, int base,
                                                 int n_total, Prep prep, Body body) {
    int nch = (n_total + kChunk - 1) / kChunk;
    if (threadIdx.x == 0) {
        for (int c = 0; c < nch && c < 2; ++c) issue_chunk(S, c, src, base, n_total);
    }
    bool ok_all = true;
    for (int ch = 0; ch < nch; ++ch) {
        int st = ch & 1;
        int n = min(kChunk, n_total - ch * kChunk);
        bool ok = mbar_wait_bounded(&S.bar[st], parity[st]);
        parity[st] ^= 1u;
        if (ok) prep(st, n);
        if (__syncthreads_or(!ok)) {
            ok_all = false;
            // let copies already in flight land before the CTA leaves
            if (threadIdx.x == 0) {
                for (int c = ch + 1; c < nch && c < ch + 2; ++c) mbar_wait_bounded(&S.bar[c & 1], parity[c & 1]);
            }
            break;
        }
        body(st, n, ch * kChunk);
        __syncthreads();
        if (threadIdx.x == 0 && ch + 2 < nch) issue_chunk(S, ch + 2, src, base, n_total);
    }
    return ok_all;
}

// Same over the chunks list[0..n_list) (in that order) only.
__device__ __forceinline__ void issue_chunk_at(Stage& S, int st, int ch, const Srcs& src, int base, int n_total) {
    int n = min(kChunk, n_total - ch * kChunk);
    uint32_t bytes = (uint32_t)n * 16u;
    mbar_expect_tx(&S.bar[st], bytes * (uint32_t)src.n);
    for (int k = 0; k < src.n; ++k) bulk_g2s(S.s[k][st], src.p[k] + base + ch * kChunk, bytes, &S.bar[st]);
}

template <class Prep, class Body>
__device__ __forceinline__ bool stream_list_prep(Stage& S, uint32_t (&parity)[2], const Srcs& src, int base,
                                                 int n_total, int n_list, Prep prep, Body body) {
    if (threadIdx.x == 0) {
        for (int c = 0; c < n_list && c < 2; ++c) issue_chunk_at(S, c & 1, S.list[c] & 0xffffff, src, base, n_total);
    }
    bool ok_all = true;
    for (int c = 0; c < n_list; ++c) {
        int st = c & 1, ch = S.list[c] & 0xffffff, mask = (int)((unsigned)S.list[c] >> 24);
        int n = min(kChunk, n_total - ch * kChunk);
        bool ok = mbar_wait_bounded(&S.bar[st], parity[st]);
        parity[st] ^= 1u;
        if (ok) prep(st, n);
        if (__syncthreads_or(!ok)) {
            ok_all = false;
            if (threadIdx.x == 0) {
                for (int k = c + 1; k < n_list && k < c + 2; ++k) mbar_wait_bounded(&S.bar[k & 1], parity[k & 1]);
            }
            break;
        }
        body(st, n, ch * kChunk, mask);
        __syncthreads();
        if (threadIdx.x == 0 && c + 2 < n_list) issue_chunk_at(S, st, S.list[c + 2] & 0xffffff, src, base, n_total);
    }
    return ok_all;
}

// ------------------------------------- exact underflow skipping (cone bounds)
// A granule is kGran pairs of one angle block (a quarter of a staged chunk); its
// cone bounds the directions of its spots: for observed spots
// the unit vectors p / |p| and the smallest |p|, for model spots the rays r
// and the largest |c|.  For an observed cone O and a model cone M, every pair
// has an angle between rhat = (p - c)/|p - c| and r of at least
//   th = angle(a_O, a_M) - beta_O - beta_M - asin(c_max / p_min)
// (the direction of p seen from c differs from p/|p| by at most
// asin(|c| / |p|)), so its cost is at least D^2 (2 sin(th/2))^2.
struct Cone {
    float ax, ay, az, beta, ext;  // axis, half-angle (rad), p_min or c_max
};

__device__ __forceinline__ Cone load_cone(const float4* cone, const float* ext, int g) {
    float4 c = cone[g];
    return Cone{c.x, c.y, c.z, c.w, ext[g]};
}

__device__ __forceinline__ float angle_between(float ax, float ay, float az, float bx, float by, float bz) {
    float c = ax * bx + ay * by + az * bz;
    return acosf(fminf(1.0f, fmaxf(-1.0f, c)));
}

// A cone containing two cones (obs: the smaller p_min, else the larger c_max).
__device__ __forceinline__ Cone merge_cones(const Cone& a, const Cone& b, bool obs) {
    float x = a.ax + b.ax, y = a.ay + b.ay, z = a.az + b.az;
    float n2 = x * x + y * y + z * z;
    Cone m;
    if (n2 < 1e-12f) {
        m = a;
        m.beta = 3.2f;  // opposite axes: no bound
    } else {
        float r = rsqrtf(n2);
        m.ax = x * r;
        m.ay = y * r;
        m.az = z * r;
        m.beta = fmaxf(angle_between(m.ax, m.ay, m.az, a.ax, a.ay, a.az) + a.beta,
                       angle_between(m.ax, m.ay, m.az, b.ax, b.ay, b.az) + b.beta) + 1e-5f;
    }
    m.ext = obs ? fminf(a.ext, b.ext) : fmaxf(a.ext, b.ext);
    return m;
}

// Lower bound of K |rhat - r|^2 (K = D^2 log2(e) / eps) over the pairs of an
// observed cone and a model cone; 0 when the cones may overlap.
__device__ __forceinline__ float min_scaled_cost(const Cone& O, const Cone& M, float K) {
    float sep = angle_between(O.ax, O.ay, O.az, M.ax, M.ay, M.az);
    float off = O.ext > M.ext ? asinf(M.ext / O.ext) : 1.6f;
    float th = sep - O.beta - M.beta - off - 1e-4f;
    if (!(th > 0.0f)) return 0.0f;
    float s = sinf(0.5f * fminf(th, 3.14159f));
    return K * 4.0f * s * s;
}

// Every plan entry of a pair whose shifted exponent is below -kSkipLog2 is
// flushed to exactly 0 by ex2.approx.ftz (below 2^-126), so the sums are
// bit-identical with or without the pair.
constexpr float kSkipLog2 = 130.0f;

// Ordered list (in Stage::list) of the chunks c < nch whose granule mask
// need(c) (bit h: granule h of the chunk can hold a plan entry) is nonzero,
// each entry c | mask << 24; returns its length.  All threads of the CTA call it.
template <class Need>
__device__ __forceinline__ int build_chunk_list(Stage& S, int nch, Need need) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int base = 0;
    for (int c0 = 0; c0 < nch; c0 += blockDim.x) {
        int c = c0 + threadIdx.x;
        int mask = c < nch ? need(c) : 0;
        bool nd = mask != 0;
        unsigned b = __ballot_sync(0xffffffffu, nd);
        if (lane == 0) S.wcnt[w] = __popc(b);
        __syncthreads();
        int before = 0, total = 0;
        for (int k = 0; k < nw; ++k) {
            if (k < w) before += S.wcnt[k];
            total += S.wcnt[k];
        }
        if (nd) S.list[base + before + __popc(b & ((1u << lane) - 1u))] = (int)((unsigned)c | ((unsigned)mask << 24));
        base += total;
        __syncthreads();
    }
    return base;
}

// Pairs of the granules of chunk ch selected by mask (n_total pairs in the block).
__device__ __forceinline__ int list_pairs(int ch, int mask, int n_total) {
    int n = min(kChunk, n_total - ch * kChunk), np = 0;
    for (int q = 0; q < kParts; ++q)
        if ((mask >> q) & 1) np += max(0, min(kGran, n - q * kGran));
    return np;
}

// Calls run(first, count) for each maximal run of selected granules of a
// staged chunk of n pairs (mask bit q: granule q).
template <class Run>
__device__ __forceinline__ void for_each_run(int mask, int n, Run run) {
    int q = 0;
    while (q < kParts) {
        if (!((mask >> q) & 1)) {
            ++q;
            continue;
        }
        int q1 = q;
        while (q1 + 1 < kParts && ((mask >> (q1 + 1)) & 1)) ++q1;
        const int h = q * kGran, e = min(n, (q1 + 1) * kGran);
        if (e > h) run(h, e - h);
        q = q1 + 1;
    }
}

// Cone of the tile's own spots [first, first + count) pairs of a block whose
// granules start at granule gb (pair offset p0): the merge of its granules.
__device__ __forceinline__ Cone tile_cone(const float4* cone, const float* ext, int gb, int p0, int first, int count,
                                          bool obs) {
    const int g0 = gb + (first - p0) / kGran, g1 = gb + (first + count - 1 - p0) / kGran;
    Cone c = load_cone(cone, ext, g0);
    for (int g = g0 + 1; g <= g1; ++g) c = merge_cones(c, load_cone(cone, ext, g), obs);
    return c;
}

// Same without a prep step.
template <class Body>
__device__ __forceinline__ bool stream_tile(Stage& S, uint32_t (&parity)[2], const Srcs& src, int base,
                                            int n_total, Body body) {
    int nch = (n_total + kChunk - 1) / kChunk;
    if (threadIdx.x == 0) {
        for (int c = 0; c < nch && c < 2; ++c) issue_chunk(S, c, src, base, n_total);
    }
    bool ok_all = true;
    for (int ch = 0; ch < nch; ++ch) {
        int st = ch & 1;
        bool ok = mbar_wait_bounded(&S.bar[st], parity[st]);
        parity[st] ^= 1u;
        if (ok) body(st, min(kChunk, n_total - ch * kChunk), ch * kChunk);
        if (__syncthreads_or(!ok)) {
            ok_all = false;
            if (threadIdx.x == 0) {
                for (int c = ch + 1; c < nch && c < ch + 2; ++c) mbar_wait_bounded(&S.bar[c & 1], parity[c & 1]);
            }
            break;
        }
        if (threadIdx.x == 0 && ch + 2 < nch) issue_chunk(S, ch + 2, src, base, n_total);
    }
    return ok_all;
}

__device__ __forceinline__ void init_stage(Stage& S) {
    if (threadIdx.x == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
}

// Tile queue: thread 0 takes the next tile index; -1 when the queue is empty.
__device__ __forceinline__ int next_tile(Stage& S, int* counter, int n_tiles) {
    if (threadIdx.x == 0) {
        int t = atomicAdd(counter, 1);
        S.tile = t < n_tiles ? t : -1;
    }
    __syncthreads();
    int t = S.tile;
    __syncthreads();
    return t;
}

// Completion ticket: true in exactly one CTA, the last one to finish.
__device__ __forceinline__ bool last_cta(Stage& S, int* done) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        int k = atomicAdd(done, 1);
        S.last = (k == (int)gridDim.x - 1);
    }
    __syncthreads();
    bool last = S.last != 0;
    if (last) __threadfence();
    return last;
}

__device__ __forceinline__ void lse_merge_into(float& m, float& s, float m2, float s2) {
    Lse2 L;
    L.m = m;
    L.s = s;
    L.merge(m2, s2);
    m = L.m;
    s = L.s;
}

// Column pair (two model spots): negated centres and rays, packed duplicates.
struct ColPair {
    f2 ncxa, ncya, ncza, nrxa, nrya, nrza;
    f2 ncxb, ncyb, nczb, nrxb, nryb, nrzb;
    f2 ka, kb;  // {-K_a, -K_a}, {-K_b, -K_b}: cost factors of the two model spots
    RowLse A, B;
};

__device__ __forceinline__ void load_col_pair(const SkArgs& a, int q, ColPair& C) {
    float4 X = a.modX[q], Y = a.modY[q], Z = a.modZ[q], W = a.modW[q];
    C.ncxa = dup(X.x);
    C.ncya = dup(X.z);
    C.ncza = dup(Y.x);
    C.nrxa = dup(Z.x);
    C.nrya = dup(Z.z);
    C.nrza = dup(W.x);
    C.ncxb = dup(X.y);
    C.ncyb = dup(X.w);
    C.nczb = dup(Y.y);
    C.nrxb = dup(Z.y);
    C.nryb = dup(Z.w);
    C.nrzb = dup(W.y);
    C.ka = dup(W.z);
    C.kb = dup(W.w);
}

}  // namespace laue
