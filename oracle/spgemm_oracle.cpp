// CPU oracle for semiring SpGEMM -- TEST INFRASTRUCTURE ONLY.
//
// This file is the slow, obviously correct definition the CUDA library is
// checked against.  Only the test suite, the smoke check and the benchmark's
// CPU-baseline leg may load it.  It shares no code, header or constant with the
// CUDA path.
//
// What it computes (McFarland, Bellavita, Guidi, ICPE'25):
//   * SpGEMM C = A (x).(+) B (Section 2.1) over a semiring whose addition (+)
//     is commutative and associative and whose multiplication (x) is
//     associative (Section 2.2).  For every row i and column j
//         C[i,j] = (+)_{k in cols(A_i), j in cols(B_k)} A[i,k] (x) B[k,j]
//     and (i,j) is stored iff at least one product exists (structural
//     pattern: no value-based pruning).  Row-wise Gustavson with an ordered
//     map per output row: k ascending over A_i, then j ascending over B_k;
//     the first product of a column initialises its accumulator, later ones
//     are folded in with (+) from the left.
//   * The semirings: plus-times over double / float / int64 (the "float"
//     semiring of the experiments, Section 4), min-plus over float (Section
//     2.2 shortest paths: (+) = min, (x) = +), boolean or-and (pattern only),
//     and the k-mer overlap semiring (genomics use, Section 1): (x) builds
//     {count 1, pair (a,b)}, (+) adds counts and keeps the two
//     lexicographically smallest pairs.
//   * The transpose used by the identity AB = (B^T A^T)^T (Section 3.1).
//   * The merge of per-stage partial products: C = (+)_s P^(s), folded in
//     stage order (Sections 2.1 and 3.4).
//
// Readings where the paper is silent: min-plus (+) is min under the IEEE
// total order restricted to non-NaN values (so -0 < +0); plus-times int64
// wraps modulo 2^64; overlap pairs compare (a, b) lexicographically and the
// empty pair is (INT32_MAX, INT32_MAX).
//
// Build: g++ -O2 -ffp-contract=off -fPIC -shared -pthread (see build.py).

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <thread>
#include <utility>
#include <vector>

namespace {

enum { SR_PT_F64 = 0, SR_BOOL = 1, SR_MP_F32 = 2, SR_OVERLAP = 3, SR_PT_I64 = 4, SR_PT_F32 = 5 };

struct OCsr {
    int64_t nrows, ncols;
    const int64_t* rp;
    const int32_t* col;
    const void* val;
};

// ---- semirings, written as plainly as possible -------------------------------

struct PtF64 {
    using In = double;
    using Acc = double;
    static Acc mul(In a, In b) { return a * b; }
    static Acc add(Acc x, Acc y) { return x + y; }
};

struct PtF32 {
    using In = float;
    using Acc = float;
    static Acc mul(In a, In b) { return a * b; }
    static Acc add(Acc x, Acc y) { return x + y; }
};

struct PtI64 {
    using In = int64_t;
    using Acc = int64_t;
    static Acc mul(In a, In b) { return (int64_t)((uint64_t)a * (uint64_t)b); }
    static Acc add(Acc x, Acc y) { return (int64_t)((uint64_t)x + (uint64_t)y); }
};

struct MpF32 {
    using In = float;
    using Acc = float;
    static Acc mul(In a, In b) { return a + b; }
    // min; on equal values prefer -0 over +0 (IEEE total order).
    static Acc add(Acc x, Acc y) {
        if (y < x) return y;
        if (x < y) return x;
        if (std::signbit(y) && !std::signbit(x)) return y;
        return x;
    }
};

struct Bool {
    using In = char;   // unused: pattern only
    using Acc = char;
    static Acc mul(In, In) { return 1; }
    static Acc add(Acc, Acc) { return 1; }
};

struct OvPair {
    int32_t a, b;
};
static bool pair_less(OvPair x, OvPair y) { return x.a < y.a || (x.a == y.a && x.b < y.b); }
static const OvPair kNoPair = {INT32_MAX, INT32_MAX};

struct OvAcc {
    int32_t count;
    OvPair p1, p2;   // p1 <= p2; kNoPair when absent
};

struct Overlap {
    using In = int32_t;
    using Acc = OvAcc;
    static Acc mul(In a, In b) { return OvAcc{1, OvPair{a, b}, kNoPair}; }
    static Acc add(const Acc& x, const Acc& y) {
        OvPair all[4] = {x.p1, x.p2, y.p1, y.p2};
        // the two smallest of four, by selection
        int m1 = 0;
        for (int t = 1; t < 4; ++t)
            if (pair_less(all[t], all[m1])) m1 = t;
        int m2 = (m1 == 0) ? 1 : 0;
        for (int t = 0; t < 4; ++t)
            if (t != m1 && pair_less(all[t], all[m2])) m2 = t;
        return OvAcc{(int32_t)((uint32_t)x.count + (uint32_t)y.count), all[m1], all[m2]};
    }
};

// output element written for each semiring
template <class S> struct Out { using T = typename S::Acc; };
struct OvOut { int32_t count, a0, b0, a1, b1; };
template <> struct Out<Overlap> { using T = OvOut; };

template <class S> static typename Out<S>::T to_out(const typename S::Acc& v) { return v; }
template <> OvOut to_out<Overlap>(const OvAcc& v) {
    return OvOut{v.count, v.p1.a, v.p1.b, v.p2.a, v.p2.b};
}
template <class S> static typename S::Acc from_out(const typename Out<S>::T& v) { return v; }
template <> OvAcc from_out<Overlap>(const OvOut& v) {
    return OvAcc{v.count, OvPair{v.a0, v.b0}, OvPair{v.a1, v.b1}};
}

// ---- result object -------------------------------------------------------------

struct Result {
    int64_t nrows = 0, ncols = 0;
    int out_bytes = 0;                         // bytes per output value (0 = pattern)
    std::vector<std::vector<int32_t>> cols;    // per selected row
    std::vector<std::vector<char>> vals;       // per selected row, raw bytes
};

template <class F>
static void parallel_rows(int64_t n, int threads, F&& body) {
    if (threads <= 1 || n < 64) {
        for (int64_t r = 0; r < n; ++r) body(r);
        return;
    }
    std::atomic<int64_t> next(0);
    const int64_t chunk = 16;
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t)
        pool.emplace_back([&]() {
            for (;;) {
                int64_t r0 = next.fetch_add(chunk);
                if (r0 >= n) break;
                int64_t r1 = r0 + chunk < n ? r0 + chunk : n;
                for (int64_t r = r0; r < r1; ++r) body(r);
            }
        });
    for (auto& th : pool) th.join();
}

template <class S>
static Result* gustavson(const OCsr& A, const OCsr& B, int64_t nsel, const int64_t* rows,
                         int threads) {
    using In = typename S::In;
    using Acc = typename S::Acc;
    using OutT = typename Out<S>::T;
    const bool pattern = std::is_same<S, Bool>::value;
    Result* R = new Result;
    R->nrows = nsel;
    R->ncols = B.ncols;
    R->out_bytes = pattern ? 0 : (int)sizeof(OutT);
    R->cols.resize(nsel);
    R->vals.resize(nsel);
    const In* av = (const In*)A.val;
    const In* bv = (const In*)B.val;
    parallel_rows(nsel, threads, [&](int64_t r) {
        const int64_t i = rows ? rows[r] : r;
        std::map<int32_t, Acc> acc;
        for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
            const int32_t k = A.col[p];
            const In a = pattern ? In() : av[p];
            for (int64_t q = B.rp[k]; q < B.rp[k + 1]; ++q) {
                const int32_t j = B.col[q];
                const Acc prod = S::mul(a, pattern ? In() : bv[q]);
                auto it = acc.find(j);
                if (it == acc.end())
                    acc.emplace(j, prod);
                else
                    it->second = S::add(it->second, prod);
            }
        }
        std::vector<int32_t>& oc = R->cols[r];
        std::vector<char>& ov = R->vals[r];
        oc.reserve(acc.size());
        if (!pattern) ov.resize(acc.size() * sizeof(OutT));
        size_t t = 0;
        for (const auto& kv : acc) {
            oc.push_back(kv.first);
            if (!pattern) {
                OutT o = to_out<S>(kv.second);
                std::memcpy(ov.data() + t * sizeof(OutT), &o, sizeof(OutT));
            }
            ++t;
        }
    });
    return R;
}

// merge: C = P^(0) (+) P^(1) (+) ... folded in stage order; values are outputs.
template <class S>
static Result* merge(int nparts, const OCsr* parts, int threads) {
    using Acc = typename S::Acc;
    using OutT = typename Out<S>::T;
    const bool pattern = std::is_same<S, Bool>::value;
    Result* R = new Result;
    R->nrows = parts[0].nrows;
    R->ncols = parts[0].ncols;
    R->out_bytes = pattern ? 0 : (int)sizeof(OutT);
    R->cols.resize(R->nrows);
    R->vals.resize(R->nrows);
    parallel_rows(R->nrows, threads, [&](int64_t i) {
        std::map<int32_t, Acc> acc;
        for (int s = 0; s < nparts; ++s) {
            const OCsr& P = parts[s];
            const OutT* pv = (const OutT*)P.val;
            for (int64_t q = P.rp[i]; q < P.rp[i + 1]; ++q) {
                const int32_t j = P.col[q];
                const Acc v = pattern ? Acc() : from_out<S>(pv[q]);
                auto it = acc.find(j);
                if (it == acc.end())
                    acc.emplace(j, v);
                else
                    it->second = S::add(it->second, v);
            }
        }
        std::vector<int32_t>& oc = R->cols[i];
        std::vector<char>& ov = R->vals[i];
        if (!pattern) ov.resize(acc.size() * sizeof(OutT));
        size_t t = 0;
        for (const auto& kv : acc) {
            oc.push_back(kv.first);
            if (!pattern) {
                OutT o = to_out<S>(kv.second);
                std::memcpy(ov.data() + t * sizeof(OutT), &o, sizeof(OutT));
            }
            ++t;
        }
    });
    return R;
}

template <template <class> class Fn, class... Args>
static Result* dispatch(int sr, Args&&... args) {
    switch (sr) {
        case SR_PT_F64: return Fn<PtF64>::run(args...);
        case SR_BOOL: return Fn<Bool>::run(args...);
        case SR_MP_F32: return Fn<MpF32>::run(args...);
        case SR_OVERLAP: return Fn<Overlap>::run(args...);
        case SR_PT_I64: return Fn<PtI64>::run(args...);
        case SR_PT_F32: return Fn<PtF32>::run(args...);
        default: return nullptr;
    }
}

template <class S> struct GustavsonFn {
    static Result* run(const OCsr* A, const OCsr* B, int64_t nsel, const int64_t* rows, int th) {
        return gustavson<S>(*A, *B, nsel, rows, th);
    }
};
template <class S> struct MergeFn {
    static Result* run(int nparts, const OCsr* parts, int th) { return merge<S>(nparts, parts, th); }
};

}  // namespace

extern "C" {

// C = A (x).(+) B restricted to the listed rows of A (rows == NULL: all rows,
// nsel must then equal A->nrows).  Returns NULL on invalid arguments.
void* oracle_spgemm_rows(int sr, const OCsr* A, const OCsr* B, int64_t nsel,
                         const int64_t* rows, int threads) {
    if (!A || !B || A->ncols != B->nrows) return nullptr;
    if (!rows && nsel != A->nrows) return nullptr;
    return dispatch<GustavsonFn>(sr, A, B, nsel, rows, threads);
}

// C = (+)_{s=0..nparts-1} parts[s], same shape for all parts, values are of the
// semiring's output type (20-byte records for the overlap semiring).
void* oracle_merge(int sr, int nparts, const OCsr* parts, int threads) {
    if (nparts < 1 || !parts) return nullptr;
    for (int s = 1; s < nparts; ++s)
        if (parts[s].nrows != parts[0].nrows || parts[s].ncols != parts[0].ncols) return nullptr;
    return dispatch<MergeFn>(sr, nparts, parts, threads);
}

// A^T with values carried (value_bytes per entry, 0 for pattern only).
void* oracle_transpose(const OCsr* A, int value_bytes) {
    Result* R = new Result;
    R->nrows = A->ncols;
    R->ncols = A->nrows;
    R->out_bytes = value_bytes;
    R->cols.resize(A->ncols);
    R->vals.resize(A->ncols);
    const char* av = (const char*)A->val;
    for (int64_t i = 0; i < A->nrows; ++i)
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
            const int32_t j = A->col[p];
            R->cols[j].push_back((int32_t)i);
            if (value_bytes)
                R->vals[j].insert(R->vals[j].end(), av + p * value_bytes,
                                  av + (p + 1) * value_bytes);
        }
    return R;
}

int64_t oracle_result_nrows(void* r) { return ((Result*)r)->nrows; }

int64_t oracle_result_nnz(void* r) {
    int64_t n = 0;
    for (auto& c : ((Result*)r)->cols) n += (int64_t)c.size();
    return n;
}

void oracle_result_copy(void* r, int64_t* rp, int32_t* col, void* val) {
    Result* R = (Result*)r;
    int64_t pos = 0;
    rp[0] = 0;
    for (int64_t i = 0; i < R->nrows; ++i) {
        const auto& c = R->cols[i];
        if (!c.empty()) std::memcpy(col + pos, c.data(), c.size() * sizeof(int32_t));
        if (R->out_bytes && val && !c.empty())
            std::memcpy((char*)val + pos * R->out_bytes, R->vals[i].data(),
                        c.size() * R->out_bytes);
        pos += (int64_t)c.size();
        rp[i + 1] = pos;
    }
}

void oracle_result_free(void* r) { delete (Result*)r; }

}  // extern "C"
