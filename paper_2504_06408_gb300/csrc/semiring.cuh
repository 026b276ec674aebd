// Semiring functors of the device path (Section 2.2: a semiring redefines the
// entry type, the multiplication (x) and the addition (+); (+) is commutative
// and associative, (x) associative).
//
// Each semiring S provides
//   In      input value type          Slot   shared-memory accumulator word
//   Out     output value type         kVal   false: pattern only (boolean)
//   kBitmap true: the dense tier needs a presence bitmap because no Slot value
//           can mark "no product yet" (plus-times: 0 is a valid sum)
//   empty()            initial Slot (the (+) identity in Slot form)
//   acc(Slot*, a, b)   atomically fold a (x) b into *Slot (order-free for the
//                      exact semirings, order-dependent rounding for floats)
//   touched(Slot)      some product reached this Slot (only when !kBitmap)
//   out(Slot)          Slot -> output value
//   prod(a, b)         a (x) b as an output value (register accumulation)
//   add(Out, Out)      plain (+) on outputs (stage merge, register accumulation)
#pragma once

#include "common.cuh"

namespace spg {

enum SemiringId : int {
    SR_PT_F64 = 0,
    SR_BOOL = 1,
    SR_MP_F32 = 2,
    SR_OVERLAP = 3,
    SR_PT_I64 = 4,
    SR_PT_F32 = 5,
};

struct SrPtF64 {
    using In = double;
    using Slot = double;
    using Out = double;
    static constexpr bool kVal = true, kBitmap = true;
    static SPG_DEV Slot empty() { return 0.0; }
    static SPG_DEV void acc(Slot* s, In a, In b) { atomicAdd(s, __dmul_rn(a, b)); }
    static SPG_DEV bool touched(Slot) { return true; }
    static SPG_DEV Out out(Slot v) { return v; }
    static SPG_DEV Out prod(In a, In b) { return __dmul_rn(a, b); }
    static SPG_DEV Out add(Out x, Out y) { return __dadd_rn(x, y); }
};

struct SrPtF32 {
    using In = float;
    using Slot = float;
    using Out = float;
    static constexpr bool kVal = true, kBitmap = true;
    static SPG_DEV Slot empty() { return 0.0f; }
    static SPG_DEV void acc(Slot* s, In a, In b) { atomicAdd(s, __fmul_rn(a, b)); }
    static SPG_DEV bool touched(Slot) { return true; }
    static SPG_DEV Out out(Slot v) { return v; }
    static SPG_DEV Out prod(In a, In b) { return __fmul_rn(a, b); }
    static SPG_DEV Out add(Out x, Out y) { return __fadd_rn(x, y); }
};

struct SrPtI64 {
    using In = int64_t;
    using Slot = unsigned long long;
    using Out = int64_t;
    static constexpr bool kVal = true, kBitmap = true;
    static SPG_DEV Slot empty() { return 0ull; }
    static SPG_DEV void acc(Slot* s, In a, In b) {
        atomicAdd(s, (unsigned long long)a * (unsigned long long)b);
    }
    static SPG_DEV bool touched(Slot) { return true; }
    static SPG_DEV Out out(Slot v) { return (Out)v; }
    static SPG_DEV Out prod(In a, In b) {
        return (Out)((unsigned long long)a * (unsigned long long)b);
    }
    static SPG_DEV Out add(Out x, Out y) {
        return (Out)((unsigned long long)x + (unsigned long long)y);
    }
};

// min-plus: floats are mapped to uint32 so that unsigned order equals the
// IEEE total order on non-NaN values (-0 < +0); atomicMin then gives an exact,
// order-free minimum.  0xFFFFFFFF (the image of the all-ones NaN) marks an
// untouched slot; no non-NaN float maps to it.
SPG_DEV uint32_t f32_to_ordered(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
SPG_DEV float ordered_to_f32(uint32_t m) {
    return __uint_as_float((m & 0x80000000u) ? (m & 0x7fffffffu) : ~m);
}

struct SrMpF32 {
    using In = float;
    using Slot = uint32_t;
    using Out = float;
    static constexpr bool kVal = true, kBitmap = false;
    static SPG_DEV Slot empty() { return 0xffffffffu; }
    // a plain atomicMin: reading the slot first to skip products that cannot
    // lower it puts a dependent shared-memory round trip on every product
    static SPG_DEV void acc(Slot* s, In a, In b) {
        atomicMin(s, f32_to_ordered(__fadd_rn(a, b)));
    }
    // as acc(); returns true if the slot was untouched before (first product)
    static SPG_DEV bool acc_first(Slot* s, In a, In b) {
        const uint32_t m = f32_to_ordered(__fadd_rn(a, b));
        const uint32_t cur = *(volatile Slot*)s;
        if (m < cur) atomicMin(s, m);
        return cur == 0xffffffffu;
    }
    static SPG_DEV bool touched(Slot v) { return v != 0xffffffffu; }
    static SPG_DEV Out out(Slot v) { return ordered_to_f32(v); }
    static SPG_DEV Out prod(In a, In b) { return __fadd_rn(a, b); }
    static SPG_DEV Out add(Out x, Out y) {
        return f32_to_ordered(y) < f32_to_ordered(x) ? y : x;
    }
};

struct SrBool {
    using In = char;
    using Slot = uint32_t;
    using Out = char;
    static constexpr bool kVal = false, kBitmap = true;
    static SPG_DEV Slot empty() { return 0u; }
    static SPG_DEV void acc(Slot*, In, In) {}
    static SPG_DEV bool touched(Slot) { return true; }
    static SPG_DEV Out out(Slot) { return 1; }
    static SPG_DEV Out prod(In, In) { return 1; }
    static SPG_DEV Out add(Out, Out) { return 1; }
};

// k-mer overlap: a pair (position in read i, position in read j) is packed as
// a << 32 | b (positions are non-negative), so unsigned order is lexicographic
// order.  m1 <= m2 hold the two smallest pairs: an insert x does
// old = atomicMin(m1, x) and then atomicMin(m2, max(old, x)); every value
// except the final m1 reaches m2 exactly once, so m2 ends as the second
// smallest of the multiset whatever the interleaving.
struct OvRecord {
    int32_t count, a0, b0, a1, b1;
};
struct OvSlot {
    unsigned long long m1, m2;
    unsigned int count, pad;
};
constexpr unsigned long long kNoPair = 0x7fffffff7fffffffull;

struct SrOverlap {
    using In = int32_t;
    using Slot = OvSlot;
    using Out = OvRecord;
    static constexpr bool kVal = true, kBitmap = false;
    static SPG_DEV Slot empty() { return OvSlot{kNoPair, kNoPair, 0u, 0u}; }
    static SPG_DEV void acc(Slot* s, In a, In b) {
        const unsigned long long x =
            ((unsigned long long)(uint32_t)a << 32) | (unsigned long long)(uint32_t)b;
        atomicAdd(&s->count, 1u);
        // x >= current second smallest: neither minimum can change
        if (x >= *(volatile unsigned long long*)&s->m2) return;
        const unsigned long long old = atomicMin(&s->m1, x);
        atomicMin(&s->m2, old > x ? old : x);
    }
    static SPG_DEV bool acc_first(Slot* s, In a, In b) {
        const unsigned long long x =
            ((unsigned long long)(uint32_t)a << 32) | (unsigned long long)(uint32_t)b;
        const unsigned int c0 = atomicAdd(&s->count, 1u);
        if (x < *(volatile unsigned long long*)&s->m2) {
            const unsigned long long old = atomicMin(&s->m1, x);
            atomicMin(&s->m2, old > x ? old : x);
        }
        return c0 == 0u;
    }
    static SPG_DEV bool touched(const Slot& v) { return v.count != 0u; }
    static SPG_DEV Out out(const Slot& v) {
        return OvRecord{(int32_t)v.count, (int32_t)(v.m1 >> 32), (int32_t)(v.m1 & 0xffffffffu),
                        (int32_t)(v.m2 >> 32), (int32_t)(v.m2 & 0xffffffffu)};
    }
    static SPG_DEV Out prod(In a, In b) { return OvRecord{1, a, b, INT32_MAX, INT32_MAX}; }
    static SPG_DEV unsigned long long pk(int32_t a, int32_t b) {
        return ((unsigned long long)(uint32_t)a << 32) | (unsigned long long)(uint32_t)b;
    }
    static SPG_DEV Out add(const Out& x, const Out& y) {
        unsigned long long p[4] = {pk(x.a0, x.b0), pk(x.a1, x.b1), pk(y.a0, y.b0), pk(y.a1, y.b1)};
        unsigned long long m1 = p[0], m2 = kNoPair;
#pragma unroll
        for (int t = 1; t < 4; ++t) {
            if (p[t] < m1) { m2 = m1; m1 = p[t]; }
            else if (p[t] < m2) m2 = p[t];
        }
        return OvRecord{(int32_t)((uint32_t)x.count + (uint32_t)y.count), (int32_t)(m1 >> 32),
                        (int32_t)(m1 & 0xffffffffu), (int32_t)(m2 >> 32),
                        (int32_t)(m2 & 0xffffffffu)};
    }
};

// The overlap semiring on positions below 2^16 (k-mer positions in reads of
// fewer than 65,536 k-mers): a pair packs into 32 bits as a << 16 | b, whose
// unsigned order is still lexicographic, so a slot is 12 bytes (count and
// the two smallest packed pairs) instead of 24, and the CTA hash tier holds
// rows of twice as many outputs.  Same (x), (+) and output record as
// SrOverlap; used only after the inputs' positions were checked on the device.
struct OvSlotC {
    unsigned int m1, m2, count;
};
constexpr unsigned int kNoPairC = 0xffffffffu;

struct SrOverlapC {
    using In = int32_t;
    using Slot = OvSlotC;
    using Out = OvRecord;
    static constexpr bool kVal = true, kBitmap = false;
    static SPG_DEV Slot empty() { return OvSlotC{kNoPairC, kNoPairC, 0u}; }
    static SPG_DEV void acc(Slot* s, In a, In b) {
        const unsigned int x = ((unsigned int)a << 16) | (unsigned int)b;
        atomicAdd(&s->count, 1u);
        if (x >= *(volatile unsigned int*)&s->m2) return;
        const unsigned int old = atomicMin(&s->m1, x);
        atomicMin(&s->m2, old > x ? old : x);
    }
    static SPG_DEV bool touched(const Slot& v) { return v.count != 0u; }
    static SPG_DEV int32_t hi(unsigned int x) { return x == kNoPairC ? INT32_MAX : (int32_t)(x >> 16); }
    static SPG_DEV int32_t lo(unsigned int x) { return x == kNoPairC ? INT32_MAX : (int32_t)(x & 0xffffu); }
    static SPG_DEV Out out(const Slot& v) {
        return OvRecord{(int32_t)v.count, hi(v.m1), lo(v.m1), hi(v.m2), lo(v.m2)};
    }
    static SPG_DEV Out prod(In a, In b) { return SrOverlap::prod(a, b); }
    static SPG_DEV Out add(const Out& x, const Out& y) { return SrOverlap::add(x, y); }
};

// Calls f.template operator()<S>() with the semiring type of a runtime id.
template <class F>
inline bool dispatch_semiring(int sr, F&& f) {
    switch (sr) {
        case SR_PT_F64: f.template operator()<SrPtF64>(); return true;
        case SR_BOOL: f.template operator()<SrBool>(); return true;
        case SR_MP_F32: f.template operator()<SrMpF32>(); return true;
        case SR_OVERLAP: f.template operator()<SrOverlap>(); return true;
        case SR_PT_I64: f.template operator()<SrPtI64>(); return true;
        case SR_PT_F32: f.template operator()<SrPtF32>(); return true;
        default: return false;
    }
}

inline int in_bytes(int sr) {
    switch (sr) {
        case SR_PT_F64: case SR_PT_I64: return 8;
        case SR_MP_F32: case SR_PT_F32: case SR_OVERLAP: return 4;
        default: return 0;
    }
}
inline int out_bytes(int sr) {
    switch (sr) {
        case SR_PT_F64: case SR_PT_I64: return 8;
        case SR_MP_F32: case SR_PT_F32: return 4;
        case SR_OVERLAP: return 20;
        default: return 0;
    }
}

}  // namespace spg
