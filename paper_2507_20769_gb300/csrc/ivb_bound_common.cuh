// ivb_bound_common.cuh -- the parts of the bounding kernel (Section 3.1) that
// do not depend on how the tape is evaluated, shared by the tape interpreter
// (ivb_kernels.cu) and the tape-specialised kernels generated and compiled at
// problem creation (ivb_jit.cpp):
//   the persistent tile loop over the node queue,
//   Step 1: decoding of subdomain X_k and its centre c from the index k,
//           dimension 0 fastest (Section 3.1.1),
//   the Mean Value Form sum of Definition 5 and the choice of the form,
//   the feasibility tests of the constraint enclosures,
//   Step 3: refinement hull by warp shuffles and ordered-integer atomics.
#pragma once
#include "ivb_internal.h"
#include "ivb_iv.cuh"
#include "ivb_kparams.h"

namespace ivb {

// ------------------------------------------------------------ reduction keys
// unsigned key with the order of the doubles (NaN maps to the given end)
__device__ __forceinline__ unsigned long long ukey(double x) {
    unsigned long long b = (unsigned long long)bits(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}
__device__ __forceinline__ unsigned long long ukey_lo(double x) {   // NaN -> -inf
    return isnan_(x) ? ukey(from_bits((long long)0xFFF0000000000000ULL)) : ukey(x);
}
__device__ __forceinline__ unsigned long long ukey_hi(double x) {   // NaN -> +inf
    return isnan_(x) ? ukey(from_bits(0x7FF0000000000000LL)) : ukey(x);
}
__device__ __forceinline__ double unkey(unsigned long long k) {
    return from_bits((long long)((k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k));
}

__device__ __forceinline__ unsigned long long shfl_xor64(unsigned long long v, int m) {
    unsigned lo = (unsigned)v, hi = (unsigned)(v >> 32);
    lo = __shfl_xor_sync(0xFFFFFFFFu, lo, m);
    hi = __shfl_xor_sync(0xFFFFFFFFu, hi, m);
    return ((unsigned long long)hi << 32) | lo;
}
__device__ __forceinline__ unsigned long long warp_min64(unsigned long long v) {
    for (int m = 16; m; m >>= 1) { unsigned long long o = shfl_xor64(v, m); v = o < v ? o : v; }
    return v;
}
__device__ __forceinline__ unsigned long long warp_max64(unsigned long long v) {
    for (int m = 16; m; m >>= 1) { unsigned long long o = shfl_xor64(v, m); v = o > v ? o : v; }
    return v;
}

// min (is_min) or max of v into *dst: one atomic per warp when every lane of
// the warp belongs to the same node, else one per lane; invalid lanes carry
// the neutral key.
__device__ __forceinline__ void reduce_key(unsigned long long* base, int node, int slot, int stride,
                                           unsigned long long v, bool valid, bool uniform, bool is_min) {
    if (uniform) {
        unsigned long long r = is_min ? warp_min64(valid ? v : ~0ULL) : warp_max64(valid ? v : 0ULL);
        if ((threadIdx.x & 31) == 0 && node >= 0) {
            if (is_min) atomicMin(base + (long long)node * stride + slot, r);
            else atomicMax(base + (long long)node * stride + slot, r);
        }
    } else if (valid) {
        if (is_min) atomicMin(base + (long long)node * stride + slot, v);
        else atomicMax(base + (long long)node * stride + slot, v);
    }
}

// ------------------------------------------------------------ tile loop
// one lane's subdomain in the tile loop
struct Sub {
    long long g;         // global subdomain index
    int node;            // node of g (-1 on an idle lane)
    unsigned int k;      // index of the subdomain inside its node
    bool valid;          // the lane has a subdomain
    bool uniform;        // every valid lane of the warp is on one node
    const char* rec;     // the node's queue record
};

// Blocks grab tiles of the global subdomain index space from a device counter
// and map indices to nodes through the queue's prefix sums; body(sub) runs
// for every lane of every pass (idle lanes included, for the warp reductions).
// `per` subdomains per pass: thread t takes subdomain g0 + t % per, so with
// per = blockDim / T the T groups of blockDim / T threads (whole warps) take
// the same subdomains (T threads per subdomain); per = blockDim otherwise.
template <class Body>
__device__ __forceinline__ void tile_loop_per(const KParams& P, const int per, Body&& body) {
    const long long* qh = reinterpret_cast<const long long*>(P.queue);
    const int n_nodes = (int)qh[0];
    const long long total = qh[1];
    const long long* off = reinterpret_cast<const long long*>(P.queue + kQueueHeader);
    const char* recs = P.queue + kQueueHeader + 8 * (long long)(n_nodes + 1);
    __shared__ long long s_base;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_base = (long long)atomicAdd(P.counter, (unsigned long long)P.tile);
        __syncthreads();
        const long long base = s_base;
        if (base >= total) break;
        const long long end = base + P.tile < total ? base + P.tile : total;
        for (long long g0 = base; g0 < end; g0 += per) {
            Sub s;
            s.g = g0 + (int)(threadIdx.x % (unsigned)per);
            s.valid = s.g < end;
            // node of g: largest node with off[node] <= g
            s.node = -1;
            s.k = 0;
            s.rec = recs;
            if (s.valid) {
                int lo = 0, hi = n_nodes - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (__ldg(off + mid) <= s.g) lo = mid; else hi = mid - 1;
                }
                s.node = lo;
                s.k = (unsigned int)(s.g - __ldg(off + lo));
                s.rec = recs + (long long)lo * P.rec_bytes;
            }
            const int node0 = __shfl_sync(0xFFFFFFFFu, s.node, 0);
            s.uniform = __all_sync(0xFFFFFFFFu, !s.valid || s.node == node0);
            body(s);
        }
    }
}

template <class Body>
__device__ __forceinline__ void tile_loop(const KParams& P, Body&& body) {
    tile_loop_per(P, (int)blockDim.x, body);
}

// the lane's subdomain g of [.., end): node by binary search over the prefix
// offsets, index inside the node, record, warp uniformity
__device__ __forceinline__ Sub make_sub(long long g, long long end, int n_nodes, const long long* off,
                                        const char* recs, int rec_bytes) {
    Sub s;
    s.g = g;
    s.valid = g < end;
    s.node = -1;
    s.k = 0;
    s.rec = recs;
    if (s.valid) {
        int lo = 0, hi = n_nodes - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(off + mid) <= g) lo = mid; else hi = mid - 1;
        }
        s.node = lo;
        s.k = (unsigned int)(g - __ldg(off + lo));
        s.rec = recs + (long long)lo * rec_bytes;
    }
    const int node0 = __shfl_sync(0xFFFFFFFFu, s.node, 0);
    s.uniform = __all_sync(0xFFFFFFFFu, !s.valid || s.node == node0);
    return s;
}

// As tile_loop_per with two subdomains per thread per pass: g0 + t % per and
// g0 + per + t % per, so a pass covers 2 per subdomains (the tile is a
// multiple of 2 per); body(s0, s1) with s1 invalid where the range ends.
template <class Body>
__device__ __forceinline__ void tile_loop_per2(const KParams& P, const int per, Body&& body) {
    const long long* qh = reinterpret_cast<const long long*>(P.queue);
    const int n_nodes = (int)qh[0];
    const long long total = qh[1];
    const long long* off = reinterpret_cast<const long long*>(P.queue + kQueueHeader);
    const char* recs = P.queue + kQueueHeader + 8 * (long long)(n_nodes + 1);
    __shared__ long long s_base2;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_base2 = (long long)atomicAdd(P.counter, (unsigned long long)P.tile);
        __syncthreads();
        const long long base = s_base2;
        if (base >= total) break;
        const long long end = base + P.tile < total ? base + P.tile : total;
        const long long lane = (long long)(threadIdx.x % (unsigned)per);
        for (long long g0 = base; g0 < end; g0 += 2 * (long long)per) {
            const Sub s0 = make_sub(g0 + lane, end, n_nodes, off, recs, P.rec_bytes);
            const Sub s1 = make_sub(g0 + per + lane, end, n_nodes, off, recs, P.rec_bytes);
            body(s0, s1);
        }
    }
}

// Step 1 for dimension i (Section 2.2 splitting item i): j = kk mod N_i, then
// kk /= N_i; endpoints lo + j h and lo + (j + 1) h (round to nearest, clamped
// to the node, the node's own ends at j = 0 and j = N_i - 1) and the centre
// RN(RN(e0 + e1) / 2).
__device__ __forceinline__ void decode_dim(const char* rec, int n, int i, unsigned int& kk, iv& X, double& c) {
    const double* rlo = reinterpret_cast<const double*>(rec);
    const int32_t* rN = reinterpret_cast<const int32_t*>(rlo + 3 * n);
    const unsigned int N = (unsigned int)__ldg(rN + i);
    const unsigned int j = kk % N;
    kk /= N;
    const double lo = __ldg(rlo + i), hi = __ldg(rlo + n + i), h = __ldg(rlo + 2 * n + i);
    double e0 = lo, e1 = hi;
    // j and j + 1 (< 2^31) converted exactly on the integer pipe
    if (j > 0) e0 = imin(imax(__dadd_rn(lo, __dmul_rn(int_to_double((int)j), h)), lo), hi);
    if (j + 1 < N) e1 = imin(imax(__dadd_rn(lo, __dmul_rn(int_to_double((int)(j + 1)), h)), lo), hi);
    X = mk(e0, e1);
    c = __dmul_rn(__dadd_rn(e0, e1), 0.5);
}

// ------------------------------------------------------- Step 2 and the tests
// one term of the Mean Value Form (Definition 5), summed left to right:
// acc + G_i (X_i - c_i), product and sum fused (one directed rounding per end)
__device__ __forceinline__ iv mvf_term(iv acc, iv Gi, iv Xi, double ci) {
    const iv dx = mk(sub_dn(Xi.lo, ci), sub_up(Xi.hi, ci));
    return iv_fma(Gi, dx, acc);
}

// enclosure of one output: MVF, NIE or their intersection; NaN -> ENTIRE
__device__ __forceinline__ iv final_form(int form, iv mvf, iv nie) {
    iv F = mvf;
    if (form == 1) F = nie;
    else if (form == 2) F = iv_meet(mvf, nie);
    if (isnan_(F.lo) || isnan_(F.hi)) F = entire();
    return F;
}

// the enclosure proves the subdomain infeasible for this constraint
__device__ __forceinline__ bool excludes_feasible(uint32_t kind, iv F) {
    return (kind == OUT_INEQ && gt0(F.lo)) || (kind == OUT_EQ && (gt0(F.lo) || lt0(F.hi)));
}

// Step 3: refinement hull of output o over the node's subdomains
__device__ __forceinline__ void reduce_output(const KParams& P, const Sub& s, int n_out, int o, iv F) {
    const int K = 2 * n_out + 2;
    reduce_key(P.keys, s.node, o, K, ukey_lo(F.lo), s.valid, s.uniform, true);
    reduce_key(P.keys, s.node, n_out + o, K, ukey_hi(F.hi), s.valid, s.uniform, false);
}

// certified-feasible centre upper bound and filtered objective minimum
__device__ __forceinline__ void reduce_extras(const KParams& P, const Sub& s, int n_out, double ub, double obj_lo) {
    const int K = 2 * n_out + 2;
    reduce_key(P.keys, s.node, 2 * n_out, K, ukey_hi(ub), s.valid, s.uniform, true);
    reduce_key(P.keys, s.node, 2 * n_out + 1, K, ukey_lo(obj_lo), s.valid, s.uniform, true);
}

}  // namespace ivb
