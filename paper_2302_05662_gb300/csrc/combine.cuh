// Joining the partial sums of a row that several work units (warp chunks,
// thread-block segments) computed, without any unit waiting for another.
//
// A row spanning exactly two units (the common case: a row crossing one
// chunk boundary) meets in a 64-bit exchange slot: each unit swaps its
// partial in; the one that finds the other's partial adds the two in unit
// order and writes y.  The slot holds the partial itself, so no memory fence
// is needed.  A row spanning three or more units leaves each partial in
// head/tail storage and counts its arrival with an acquire-release atomic;
// the last unit to arrive adds all partials in unit order.  Either way the sum order is fixed, so
// results do not depend on scheduling, and every slot and counter is
// restored by the unit that consumes it.
#pragma once

#include "internal.cuh"

namespace spmv {

template <typename T>
struct PartialsT {
    T *head;
    T *tail;
    unsigned *count;
    unsigned long long *xslot;
    int stride;
    static PartialsT of(const Partials &p) {
        return PartialsT{(T *)p.head, (T *)p.tail, p.count, p.xslot, p.stride};
    }
};

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

template <typename T> struct XEnc;
template <> struct XEnc<double> {
    // a signalling NaN: arithmetic never produces this bit pattern
    static constexpr unsigned long long EMPTY = 0x7FF00000DEADBEEFull;
    static __device__ __forceinline__ unsigned long long enc(double v) {
        return (unsigned long long)__double_as_longlong(v);
    }
    static __device__ __forceinline__ double dec(unsigned long long b) { return __longlong_as_double((long long)b); }
};
template <> struct XEnc<float> {
    static constexpr unsigned long long EMPTY = 0ull;  // a tag bit marks a full slot
    static __device__ __forceinline__ unsigned long long enc(float v) {
        return (1ull << 32) | (unsigned long long)__float_as_uint(v);
    }
    static __device__ __forceinline__ float dec(unsigned long long b) { return __uint_as_float((unsigned)b); }
};

// Unit c contributes `contrib` to a row spanning units c0..c1 (c0 < c1);
// `off` selects the row among `stride` rows sharing the units.  Returns true
// (with the row total) for the one arrival that completes the row.
template <typename T>
__device__ __forceinline__ bool join_partial(int64_t c, int64_t c0, int64_t c1, int off, T contrib,
                                          const PartialsT<T> &P, T *total) {
    const int64_t st = P.stride;
    if (c1 == c0 + 1) {
        unsigned long long *slot = P.xslot + c0 * st + off;
        const unsigned long long old = atomicExch(slot, XEnc<T>::enc(contrib));
        if (old == XEnc<T>::EMPTY) return false;
        const T other = XEnc<T>::dec(old);
        *total = (c == c0) ? contrib + other : other + contrib;
        *slot = XEnc<T>::EMPTY;
        return true;
    }
    if (c == c0) P.tail[c * st + off] = contrib;
    else P.head[c * st + off] = contrib;
    // acquire-release arrival: releases this unit's partial (stored just
    // above by this thread) and, for the last arrival, acquires every other
    // unit's partial -- no full memory fence needed
    const unsigned old = atom_add_acq_rel(P.count + c0 * st + off, 1u);
    if (old != (unsigned)(c1 - c0)) return false;
    T t = __ldcg(P.tail + c0 * st + off);
    for (int64_t k = c0 + 1; k <= c1; ++k) t += __ldcg(P.head + k * st + off);
    P.count[c0 * st + off] = 0u;
    *total = t;
    return true;
}

}  // namespace spmv
