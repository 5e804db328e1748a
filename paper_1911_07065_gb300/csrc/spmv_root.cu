// Fused CSR SpMV + root update: one pass over A per root of the GMRES
// polynomial (Algorithm 1: phi(A) v, Algorithm 3: p(A) v), plus the plain
// SpMV and the residual b - A x.  Two kernels with the same arithmetic
// (each row summed in stored order, one fused multiply-add per nonzero,
// acc = fma(val, x[col], acc), then the same epilogue), so their results
// are bit-identical:
//
// k_spmv_step, for a matrix streamed from HBM: a CTA owns a tile of rows
// (256 in FP64, 512 in FP32: two per thread).  It copies the tile's column
// indices and values into shared memory with asynchronous, coalesced
// 16-byte copies (consecutive threads take consecutive granules, so short
// rows of 5-7 entries leave no lane idle), then each thread walks its rows
// and applies the root update in the epilogue, reading and writing the
// row-aligned vectors once, coalesced.  Tiles whose nonzeros exceed the
// staging buffer are processed in chunks, so any row length is handled.
//
// k_spmv_direct, for small systems and for a matrix held in L2: one row per
// thread, its first entries read straight into registers before the wait on
// the previous step (no staging round trip).
//
// GB300 executes about two FP64 operations per clock per SM, so in FP64 the
// multiply-adds, not only the bytes, bound these kernels: one FMA per
// nonzero is the minimum and the epilogues use fused forms.
//
// Consecutive steps overlap: each is launched as a programmatic dependent of
// the previous one and reads its share of the matrix before it waits for the
// previous step's vectors.
//
// L2 policy: when the matrix and the chain's vectors fit in L2, the matrix is
// read with an evict-last hint into a set-aside and stays resident across
// the roots of a chain (every root reads the same A).  Otherwise a chain
// holds the nonzeros of its leading rows that way in a 48 MB set-aside and
// streams the rest with evict-first, prefetching it into L2 half a resident
// wave ahead.
#include <atomic>

#include "ppg_common.cuh"

namespace ppg {

constexpr int SPMV_ROWS = 256;      // threads per CTA

__device__ __forceinline__ uint64_t l2_policy(int keep) {
    uint64_t p;
    if (keep)
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    else
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, uint64_t pol) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], %2, %3;" ::"r"(s),
                 "l"(gmem), "n"(BYTES), "l"(pol)
                 : "memory");
}

// Hint: bring [b, e) into L2 (16-byte granules inside the range; nothing
// waits on it).  Both ends are rounded down to 16 bytes, which stays inside
// the (at least 256-byte aligned) allocation that holds the range.
__device__ __forceinline__ void prefetch_l2(const void* b, const void* e) {
    const uintptr_t lo = (uintptr_t)b & ~(uintptr_t)15;
    const uintptr_t hi = (uintptr_t)e & ~(uintptr_t)15;
    if (hi > lo)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo))
                     : "memory");
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, uint64_t pol) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem),
                 "l"(pol)
                 : "memory");
}

// Stage elements [c0, c1) of src into shared memory as dst[k - base], with
// base = c0 rounded down to a multiple of 4 elements.  With src 16-byte
// aligned, the 16-byte granules of [base, c1 rounded down to 4) move with one
// cp.async each (the few elements before c0 come along) and the ragged end
// per element, so nothing at or past c1 is read; otherwise every element of
// [c0, c1) is copied alone.  dst (16-byte aligned) holds c1 - base elements.
template <typename E>
__device__ __forceinline__ void stage_async(E* dst, const E* src, int32_t base, int32_t c0,
                                            int32_t c1, int tid, int nthr, uint64_t pol) {
    constexpr int PER = 16 / (int)sizeof(E);
    int32_t t0 = c0;
    if (((uintptr_t)src & 15) == 0) {
        const int32_t vend = c1 & ~3;
        const int32_t nvec = vend > base ? (vend - base) / PER : 0;
        for (int32_t q = tid; q < nvec; q += nthr) cp_async16(dst + q * PER, src + base + q * PER, pol);
        t0 = max(vend, c0);
    }
    for (int32_t k = t0 + tid; k < c1; k += nthr) cp_async<sizeof(E)>(dst + (k - base), src + k, pol);
}

// Stage a chunk of values and column indices by 16-byte granules from
// base = c0 & ~3 (measured faster than per-element copies in both precisions:
// FP64 2-D 1000^2 chains -2.6 %, 3-D 160^3 -5 %; FP32 3-D 160^3 chains -8 %).
template <typename T>
__device__ __forceinline__ void stage_chunk(T* sval, int32_t* scol, const T* vals,
                                            const int32_t* colind, int32_t base, int32_t c0,
                                            int32_t c1, int tid, int nthr, uint64_t pol) {
    stage_async<T>(sval, vals, base, c0, c1, tid, nthr, pol);
    stage_async<int32_t>(scol, colind, base, c0, c1, tid, nthr, pol);
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// The epilogue of one row: the root update of the step, given s = (A x)[r]
// and the row's inputs e0 = a0[r], e1 = a1[r], e2 = a2[r].
template <typename T, int OP>
__device__ __forceinline__ void step_epilogue(const StepArgs<T>& a, int64_t r, T s, T e0, T e1,
                                              T e2, double& sq) {
    if constexpr (OP == OP_SPMV) {
        a.o0[r] = s;
    } else if constexpr (OP == OP_RESID) {
        const T v = e0 - s;
        a.o0[r] = v;
        sq += (double)v * (double)v;
    } else if constexpr (OP == OP_PHI_REAL) {
        const T pin = fma(-a.c1, s, e0);
        a.o0[r] = (a.flags & F_FINAL) ? e2 - pin : pin;
    } else if constexpr (OP == OP_PHI_PAIR2) {
        // pi' = pi + c2 (A prod - 2a prod)
        const T t = fma(-a.c1, e0, s);
        const T pin = fma(a.c2, t, e1);
        a.o0[r] = (a.flags & F_FINAL) ? e2 - pin : pin;
    } else if constexpr (OP == OP_P_REAL) {
        const T pnew = (a.flags & F_PZERO) ? a.c1 * e0 : fma(a.c1, e0, e1);
        const T prodn = fma(-a.c1, s, e0);
        if (a.flags & F_FINAL) {
            a.o0[r] = fma(a.c3, prodn, pnew);
        } else {
            a.o0[r] = pnew;
            a.o1[r] = prodn;
        }
    } else if constexpr (OP == OP_P_PAIR1) {
        const T tmp = fma(a.c1, e0, -s);
        a.o0[r] = (a.flags & F_PZERO) ? a.c2 * tmp : fma(a.c2, tmp, e1);
        if (!(a.flags & F_NO_O1)) a.o1[r] = tmp;
    } else if constexpr (OP == OP_P_PAIR2) {
        const T prodn = fma(-a.c2, s, e0);
        if (a.flags & F_FINAL) {
            a.o0[r] = fma(a.c3, prodn, e1);
        } else {
            a.o0[r] = prodn;
        }
    }
}

// Rows per thread: FP32 tiles take two rows per thread (512 rows per CTA),
// so each CTA's latency-bound phases (row pointers, staging, gathers) serve
// twice the bytes; FP64 keeps one (at 32 registers, 2048 threads per SM).
template <typename T>
__host__ __device__ constexpr int step_rpt() { return sizeof(T) == 4 ? 2 : 1; }

// Threads per CTA of the staged step: FP64 128 (tiles of 128 rows, 16 CTAs
// per SM; 3-D 160^3 FP64 chains 6220 -> 6390 GB/s against 256, 6070 with
// 64), FP32 256 (tiles of 512 rows; 128 threads measured the same)
template <typename T>
__host__ __device__ constexpr int step_threads() { return sizeof(T) == 4 ? 256 : 128; }

// Nonzeros staged per chunk: FP64 1024 (128 rows of up to 8); FP32 3584, so
// that a tile of 512 rows of a 7-point stencil is one chunk and the CTA's
// 30.7 KB of shared memory lets 7 CTAs share an SM (with 4096, 6 fit:
// 3-D 160^3 FP32 chains 1 % slower).  Longer tiles take several chunks.
template <typename T>
__host__ __device__ constexpr int step_chunk() { return sizeof(T) == 4 ? 3584 : 1024; }

// CTAs per SM the register budget must allow (FP32: 32 registers instead
// of 40; FP64: 16 CTAs of 128 threads, 32 registers).  The FP32 second step of a pair of
// Algorithm 1 (not on the precision form's path, which applies p(A) only)
// keeps 40 registers and 6 CTAs: at 32 it spills.
template <typename T, int OP>
__host__ __device__ constexpr int step_min_ctas() {
    return sizeof(T) == 4 ? (OP == OP_PHI_PAIR2 ? 6 : 7) : 16;
}

// one row's multiply-adds over its staged nonzeros [lo, hi): four gathers in
// flight, then the last 1-3 (FP32: issued together; FP64: one at a time)
template <typename T, bool WIDE_TAIL>
__device__ __forceinline__ T row_dot(const T* sval, const int32_t* scol, const T* __restrict__ x,
                                     int32_t k, int32_t hi, T acc) {
    for (; k + 4 <= hi; k += 4) {
        const T v0 = sval[k], v1 = sval[k + 1], v2 = sval[k + 2], v3 = sval[k + 3];
        const T x0 = __ldg(x + scol[k]), x1 = __ldg(x + scol[k + 1]);
        const T x2 = __ldg(x + scol[k + 2]), x3 = __ldg(x + scol[k + 3]);
        acc = fma(v0, x0, acc);
        acc = fma(v1, x1, acc);
        acc = fma(v2, x2, acc);
        acc = fma(v3, x3, acc);
    }
    const int rem = hi - k;
    if constexpr (!WIDE_TAIL) {
#pragma unroll 1
        for (; k < hi; ++k) acc = fma(sval[k], __ldg(x + scol[k]), acc);
    } else if (rem > 0) {
        const T v0 = sval[k];
        const T x0 = __ldg(x + scol[k]);
        T v1 = T(0), x1 = T(0), v2 = T(0), x2 = T(0);
        if (rem > 1) {
            v1 = sval[k + 1];
            x1 = __ldg(x + scol[k + 1]);
        }
        if (rem > 2) {
            v2 = sval[k + 2];
            x2 = __ldg(x + scol[k + 2]);
        }
        acc = fma(v0, x0, acc);
        if (rem > 1) acc = fma(v1, x1, acc);
        if (rem > 2) acc = fma(v2, x2, acc);
    }
    return acc;
}

// PF: prefetch the tile a.pf_ahead tiles ahead (half a resident wave) into
// L2 (launched when the matrix is not held in an L2 set-aside)
template <typename T, int OP, bool PF>
__global__ void __launch_bounds__(step_threads<T>(), step_min_ctas<T, OP>())
k_spmv_step(const StepArgs<T> a) {
    constexpr int NT = step_threads<T>();      // threads per CTA
    // staging copies start at a chunk base rounded down to 4 elements
    constexpr int PAD = 4;
    constexpr int RPT = step_rpt<T>();
    constexpr int ROWS = NT * RPT;      // rows per CTA
    constexpr int CHUNK = step_chunk<T>();     // nonzeros staged per chunk
    __shared__ __align__(16) T sval[CHUNK + PAD];
    __shared__ __align__(16) int32_t scol[CHUNK + PAD];
    __shared__ int32_t srp[ROWS + 1];
    __shared__ double sred[NT / 32];

    const int64_t row0 = (int64_t)blockIdx.x * ROWS;
    const int tid = threadIdx.x;
    const int nrows = (int)(((int64_t)a.n - row0) < ROWS ? ((int64_t)a.n - row0) : ROWS);
    // L2 hint of the staging copies: evict-last for a matrix held in L2 (all
    // of it, or the leading rows), else evict-first (the policy is created
    // at each use, so that it holds no registers across the kernel)
    const bool keep = (a.flags & F_KEEP_A) || row0 < a.keep_rows;
    // Programmatic dependent launch: the next step in the stream may start
    // now; everything up to griddepcontrol.wait reads only the matrix, which
    // no step writes, so it overlaps the previous step's tail.
    asm volatile("griddepcontrol.launch_dependents;");
    // the tile that a CTA half a resident wave later stages: its nonzero
    // range is read now, beside this tile's row pointers.  CTAs near the end
    // of the grid prefetch the matrix tiles at the start of the next step
    // instead (a chain's next step reads the same matrix).
    int64_t prow = row0 + (int64_t)a.pf_ahead * ROWS;
    const bool wrap = prow >= a.n;
    if (wrap) prow -= (int64_t)gridDim.x * ROWS;
    const bool pf = PF && tid == 0 && a.pf_ahead > 0 && prow >= 0 && prow < a.n;
    const int64_t prow1 = min(prow + ROWS, (int64_t)a.n);
    int32_t pk0 = 0, pk1 = 0;
    if (pf) {
        pk0 = __ldg(a.rowptr + prow);
        pk1 = __ldg(a.rowptr + prow1);
    }
    for (int i = tid; i <= nrows; i += NT) srp[i] = __ldg(a.rowptr + row0 + i);
    __syncthreads();
    const int32_t k0 = srp[0];
    const int32_t k1 = srp[nrows];
    // thread tid owns rows tid and (RPT = 2) tid + NT of the tile
    int32_t my_lo[RPT], my_hi[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int t = tid + q * NT;
        my_lo[q] = (t < nrows) ? srp[t] : k1;
        my_hi[q] = (t < nrows) ? srp[t + 1] : k1;
    }
    // element k of the current chunk sits at sval / scol [k - base], base =
    // c0 & ~3
    {
        const int32_t c1 = min(k1, k0 + CHUNK);
        const int32_t base = k0 & ~3;
        stage_chunk<T>(sval, scol, a.vals, a.colind, base, k0, c1, tid, NT,
                       l2_policy(keep));
    }
    if (pf) {
        if (prow >= a.keep_rows) {   // (the leading rows' nonzeros are held in L2)
            prefetch_l2(a.vals + pk0, a.vals + pk1);
            prefetch_l2(a.colind + pk0, a.colind + pk1);
        }
        // and its row pointers, which the CTA reads first, before anything
        // else can start (3-D 160^3 FP32 chains -4 %)
        prefetch_l2(a.rowptr + prow, a.rowptr + prow1 + 1);
    }
    // the vectors written by the previous step are complete and visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (pf && !wrap) {
        prefetch_l2(a.x + prow, a.x + prow1);
        if (a.a0) prefetch_l2(a.a0 + prow, a.a0 + prow1);
        if (a.a1 && !(a.flags & F_PZERO)) prefetch_l2(a.a1 + prow, a.a1 + prow1);
        if (a.a2 && (a.flags & F_FINAL)) prefetch_l2(a.a2 + prow, a.a2 + prow1);
    }

    // The epilogue's row-aligned inputs do not depend on the product: load
    // them now, so their latency overlaps the staging and the gathers.
    T e0[RPT], e1[RPT], e2[RPT], acc[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        e0[q] = e1[q] = e2[q] = acc[q] = T(0);
        const int t = tid + q * NT;
        if (t < nrows) {
            const int64_t rr = row0 + t;
            if (a.a0) e0[q] = __ldg(a.a0 + rr);
            if (a.a1 && !(a.flags & F_PZERO)) e1[q] = a.a1[rr];
            if (a.a2 && (a.flags & F_FINAL)) e2[q] = __ldg(a.a2 + rr);
        }
    }

    for (int32_t c0 = k0; c0 < k1; c0 += CHUNK) {
        const int32_t c1 = min(k1, c0 + CHUNK);
        const int32_t base = c0 & ~3;
        if (c0 != k0) {   // the first chunk was issued before the wait
            stage_chunk<T>(sval, scol, a.vals, a.colind, base, c0, c1, tid, NT,
                           l2_policy(keep));
        }
        cp_async_wait_all();
        __syncthreads();
        // exactly one FMA per nonzero (GB300 issues two FP64 operations per
        // clock per SM); summation stays in column order within each row.
        // The last 1-3 nonzeros: FP32 issues their gathers together; FP64
        // takes them one at a time (the wider form took 40 registers, 6
        // instead of 8 CTAs per SM, and measured 13 % slower on 2-D chains).
        if constexpr (RPT == 1) {
            const int32_t lo = max(my_lo[0], c0) - base;
            const int32_t hi = min(my_hi[0], c1) - base;
            acc[0] = row_dot<T, sizeof(T) == 4>(sval, scol, a.x, lo, hi, acc[0]);
        } else {
            // two rows: their four-wide batches in lockstep (eight gathers
            // in flight), then each row's remainder
            int32_t ka = max(my_lo[0], c0) - base, kb = max(my_lo[1], c0) - base;
            const int32_t ha = min(my_hi[0], c1) - base, hb = min(my_hi[1], c1) - base;
            for (; ka + 4 <= ha && kb + 4 <= hb; ka += 4, kb += 4) {
                const T va0 = sval[ka], va1 = sval[ka + 1], va2 = sval[ka + 2], va3 = sval[ka + 3];
                const T vb0 = sval[kb], vb1 = sval[kb + 1], vb2 = sval[kb + 2], vb3 = sval[kb + 3];
                const T xa0 = __ldg(a.x + scol[ka]), xa1 = __ldg(a.x + scol[ka + 1]);
                const T xa2 = __ldg(a.x + scol[ka + 2]), xa3 = __ldg(a.x + scol[ka + 3]);
                const T xb0 = __ldg(a.x + scol[kb]), xb1 = __ldg(a.x + scol[kb + 1]);
                const T xb2 = __ldg(a.x + scol[kb + 2]), xb3 = __ldg(a.x + scol[kb + 3]);
                acc[0] = fma(va3, xa3, fma(va2, xa2, fma(va1, xa1, fma(va0, xa0, acc[0]))));
                acc[1] = fma(vb3, xb3, fma(vb2, xb2, fma(vb1, xb1, fma(vb0, xb0, acc[1]))));
            }
            acc[0] = row_dot<T, true>(sval, scol, a.x, ka, ha, acc[0]);
            acc[1] = row_dot<T, true>(sval, scol, a.x, kb, hb, acc[1]);
        }
        // the staged chunk is read by every thread: a barrier before it is
        // overwritten, none after the last one (3-D 160^3 chains +0.2 %)
        if (c0 + CHUNK < k1) __syncthreads();
    }

    double sq = 0.0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int t = tid + q * NT;
        if (t < nrows) step_epilogue<T, OP>(a, row0 + t, acc[q], e0[q], e1[q], e2[q], sq);
    }
    if constexpr (OP == OP_RESID) {
        // deterministic block reduction of ||r||^2
        for (int off = 16; off > 0; off >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, off);
        if ((tid & 31) == 0) sred[tid >> 5] = sq;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < NT / 32; ++w) t += sred[w];
            a.part[blockIdx.x] = t;
        }
    }
}

// Direct-read step: the same step, one row per thread, the row's matrix
// entries read straight into registers (up to PRE of them) before the wait
// on the previous step -- no shared-memory staging round, so the latency
// chain of a step is row pointers -> (wait) -> gathers -> epilogue.  Each
// row is summed in stored order with one FMA per nonzero and the same
// epilogue as k_spmv_step: bit-identical results.  Two uses:
// * small systems (PRE = 8, no register bound, CTAs of DIRECT_SMALL_ROWS
//   rows): a step is a handful of CTAs, and latency, not bytes, sets its
//   time;
// * a matrix held in L2 (F_KEEP_A; PRE = 3 or 4 and 32 registers, 8 CTAs
//   per SM; the preloads carry the evict-last hint): the staging round trip
//   is then the longer path.  2-D 1000^2 FP64 chains 57.3 -> 55.2 ms.
// MINB: minimum CTAs per SM given to __launch_bounds__ (0: no register bound).
// One row per thread of any CTA size up to SPMV_ROWS; the residual's partial
// sums are one per CTA.
template <typename T>
__device__ __forceinline__ T ld_hint(const T* p, uint64_t pol);
template <>
__device__ __forceinline__ double ld_hint<double>(const double* p, uint64_t pol) {
    double v;
    asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
template <>
__device__ __forceinline__ float ld_hint<float>(const float* p, uint64_t pol) {
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
template <>
__device__ __forceinline__ int32_t ld_hint<int32_t>(const int32_t* p, uint64_t pol) {
    int32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

constexpr int DIRECT_SMALL_ROWS = 64;   // rows (threads) per CTA for small systems
constexpr int DIRECT_L2_ROWS = 128;     // ... and for a matrix held in L2

template <typename T, int OP, int PRE, int MINB, bool HINT>
__global__ void __launch_bounds__(SPMV_ROWS, MINB)
k_spmv_direct(const StepArgs<T> a) {
    __shared__ double sred[SPMV_ROWS / 32];
    const int tid = threadIdx.x;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + tid;
    const bool live = r < a.n;
    asm volatile("griddepcontrol.launch_dependents;");
    int32_t k0 = 0, k1 = 0;
    T pv[PRE];
    int32_t pc[PRE];
    if (live) {
        k0 = __ldg(a.rowptr + r);
        k1 = __ldg(a.rowptr + r + 1);
#pragma unroll
        for (int q = 0; q < PRE; ++q) {
            if (k0 + q < k1) {
                if constexpr (HINT) {
                    pv[q] = ld_hint<T>(a.vals + k0 + q, l2_policy(1));
                    pc[q] = ld_hint<int32_t>(a.colind + k0 + q, l2_policy(1));
                } else {
                    pv[q] = __ldg(a.vals + k0 + q);
                    pc[q] = __ldg(a.colind + k0 + q);
                }
            }
        }
    }
    // the vectors written by the previous step are complete and visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    double sq = 0.0;
    if (live) {
        const T e0 = a.a0 ? __ldg(a.a0 + r) : T(0);
        const T e1 = (a.a1 && !(a.flags & F_PZERO)) ? a.a1[r] : T(0);
        const T e2 = (a.a2 && (a.flags & F_FINAL)) ? __ldg(a.a2 + r) : T(0);
        T xg[PRE];
#pragma unroll
        for (int q = 0; q < PRE; ++q)
            if (k0 + q < k1) xg[q] = __ldg(a.x + pc[q]);
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < PRE; ++q)
            if (k0 + q < k1) acc = fma(pv[q], xg[q], acc);
        // (entries past PRE without the hint: mostly in the lines the hinted
        // loads already brought in)
        for (int32_t k = k0 + PRE; k < k1; ++k)
            acc = fma(__ldg(a.vals + k), __ldg(a.x + __ldg(a.colind + k)), acc);
        step_epilogue<T, OP>(a, r, acc, e0, e1, e2, sq);
    }
    if constexpr (OP == OP_RESID) {
        for (int off = 16; off > 0; off >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, off);
        if ((tid & 31) == 0) sred[tid >> 5] = sq;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sred[w];
            a.part[blockIdx.x] = t;
        }
    }
}

// A root step whose operator product s = (M x)[r] was computed beforehand
// (M a composite operator such as phi_1(A)): the same epilogue as the
// fused kernel, one thread per row.
template <typename T, int OP>
__global__ void __launch_bounds__(SPMV_ROWS)
k_ew_step(const StepArgs<T> a, const T* __restrict__ prodv) {
    __shared__ double sred[SPMV_ROWS / 32];
    const int tid = threadIdx.x;
    const int64_t r = (int64_t)blockIdx.x * SPMV_ROWS + tid;
    const bool live = r < a.n;
    double sq = 0.0;
    if (live) {
        const T e0 = a.a0 ? __ldg(a.a0 + r) : T(0);
        const T e1 = (a.a1 && !(a.flags & F_PZERO)) ? a.a1[r] : T(0);
        const T e2 = (a.a2 && (a.flags & F_FINAL)) ? __ldg(a.a2 + r) : T(0);
        step_epilogue<T, OP>(a, r, __ldg(prodv + r), e0, e1, e2, sq);
    }
    if constexpr (OP == OP_RESID) {
        for (int off = 16; off > 0; off >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, off);
        if ((tid & 31) == 0) sred[tid >> 5] = sq;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < SPMV_ROWS / 32; ++w) t += sred[w];
            a.part[blockIdx.x] = t;
        }
    }
}

template <typename T>
int32_t launch_ew_step(int op, const StepArgs<T>& a, const T* prodv, cudaStream_t s) {
    if (a.n <= 0) return 0;
    const int grid = (a.n + SPMV_ROWS - 1) / SPMV_ROWS;
    switch (op) {
        case OP_RESID: k_ew_step<T, OP_RESID><<<grid, SPMV_ROWS, 0, s>>>(a, prodv); break;
        case OP_PHI_REAL: k_ew_step<T, OP_PHI_REAL><<<grid, SPMV_ROWS, 0, s>>>(a, prodv); break;
        case OP_PHI_PAIR2: k_ew_step<T, OP_PHI_PAIR2><<<grid, SPMV_ROWS, 0, s>>>(a, prodv); break;
        case OP_P_REAL: k_ew_step<T, OP_P_REAL><<<grid, SPMV_ROWS, 0, s>>>(a, prodv); break;
        case OP_P_PAIR1: k_ew_step<T, OP_P_PAIR1><<<grid, SPMV_ROWS, 0, s>>>(a, prodv); break;
        case OP_P_PAIR2: k_ew_step<T, OP_P_PAIR2><<<grid, SPMV_ROWS, 0, s>>>(a, prodv); break;
        default: return PPG_ERR_ARG;
    }
    ++g_launches;
    int32_t rc = check_launch("k_ew_step");
    return rc < 0 ? rc : grid;
}

template int32_t launch_ew_step<double>(int, const StepArgs<double>&, const double*,
                                        cudaStream_t);

// An upper bound on the partial sums a residual step of n rows writes (one
// per CTA): the smallest tile of any kernel that computes one (the staged
// FP64 step's 128 rows; the direct step's residual keeps 256-row CTAs)
int32_t spmv_grid_blocks(int32_t n) {
    constexpr int r64 = step_threads<double>() * step_rpt<double>();
    constexpr int r32 = step_threads<float>() * step_rpt<float>();
    constexpr int rmin = r64 < r32 ? (r64 < SPMV_ROWS ? r64 : SPMV_ROWS) : (r32 < SPMV_ROWS ? r32 : SPMV_ROWS);
    return (int32_t)(((int64_t)n + rmin - 1) / rmin);
}

// Reserve L2 for evict-last (persisting) lines on the current device: without
// a set-aside the evict-last hint is treated as normal.  This is a limit of
// this process's context on that device; it ends with the process.  A
// chain over a matrix too large for L2 sets it to kPartialL2 instead
// (set_l2_exact).  Returns the set-aside now in place.
constexpr int kL2Devices = 64;
static std::atomic<size_t> g_l2_reserved[kL2Devices];   // set-aside in place
static std::atomic<size_t> g_l2_asked[kL2Devices];      // what set_l2_exact asked for
static std::atomic<int> g_l2_bytes[kL2Devices];

static int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kL2Devices) {
        cudaGetLastError();
        return -1;
    }
    return dev;
}

static size_t reserve_l2_for(int dev, size_t bytes) {
    const size_t have = g_l2_reserved[dev].load(std::memory_order_relaxed);
    if (bytes <= have) return have;
    int maxp = 0;
    if (cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess ||
        maxp <= 0) {
        cudaGetLastError();
        return have;
    }
    const size_t want = bytes < (size_t)maxp ? bytes : (size_t)maxp;
    size_t got = have;
    if (want > have && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) == cudaSuccess &&
        cudaDeviceGetLimit(&got, cudaLimitPersistingL2CacheSize) == cudaSuccess) {
        g_l2_reserved[dev].store(got, std::memory_order_relaxed);
        g_l2_asked[dev].store(0, std::memory_order_relaxed);
    }
    cudaGetLastError();
    return g_l2_reserved[dev].load(std::memory_order_relaxed);
}

// Set the set-aside to `bytes` exactly (shrinking or growing it; persisting
// lines back to normal first).  Returns the set-aside now in place (the
// driver rounds the request to its granularity).
static size_t set_l2_exact(int dev, size_t bytes) {
    const size_t have = g_l2_reserved[dev].load(std::memory_order_relaxed);
    if (g_l2_asked[dev].load(std::memory_order_relaxed) == bytes) return have;
    int maxp = 0;
    if (cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess ||
        maxp <= 0) {
        cudaGetLastError();
        return have;
    }
    const size_t want = bytes < (size_t)maxp ? bytes : (size_t)maxp;
    cudaCtxResetPersistingL2Cache();
    size_t got = have;
    if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) == cudaSuccess &&
        cudaDeviceGetLimit(&got, cudaLimitPersistingL2CacheSize) == cudaSuccess) {
        g_l2_reserved[dev].store(got, std::memory_order_relaxed);
        g_l2_asked[dev].store(bytes, std::memory_order_relaxed);
    }
    cudaGetLastError();
    return g_l2_reserved[dev].load(std::memory_order_relaxed);
}

// Set-aside a chain over a matrix too large for L2 holds its leading rows in.
// Measured on the 3-D 160^3 chains with an unused set-aside (FP32 / FP64
// GB/s): none 6032 / 6150, 48 MB 6018 / 6147, 67 MB 5357 / 6032, 80 MB
// 4646 / 5604: up to about 48 MB the streamed part loses next to nothing.
constexpr size_t kPartialL2 = (size_t)48 << 20;

int keep_a_flag(int64_t n, int64_t nnz, int elem, int nvec, bool may_reserve,
                int32_t* keep_rows) {
    if (keep_rows) *keep_rows = 0;
    const int dev = current_device();
    if (dev < 0) return 0;
    int l2 = g_l2_bytes[dev].load(std::memory_order_relaxed);
    if (l2 == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = -1;
        }
        g_l2_bytes[dev].store(v, std::memory_order_relaxed);
        l2 = v;
    }
    if (l2 <= 0 || n <= 0) return 0;
    const double a_bytes = (double)nnz * (elem + 4) + 4.0 * (n + 1);
    const double bytes = a_bytes + (double)nvec * n * elem;
    if (!(bytes <= 0.8 * (double)l2)) {
        // streaming: a chain holds the nonzeros of its leading rows in a
        // set-aside of kPartialL2 (shrinking a larger one that an L2-resident
        // workload left: an unused 76 MB set-aside cost the 160^3 FP32 chains
        // 11 %), and streams the rest
        if (!keep_rows) return 0;
        const size_t have = may_reserve ? set_l2_exact(dev, kPartialL2)
                                        : g_l2_reserved[dev].load(std::memory_order_relaxed);
        const double rows = 0.9 * (double)have / (a_bytes / (double)n);
        *keep_rows = (int32_t)(rows < (double)n ? rows : (double)n);
        return 0;
    }
    const size_t need = (size_t)(a_bytes * 1.05);
    if (may_reserve) {
        reserve_l2_for(dev, need);
        return F_KEEP_A;
    }
    // no change to the context: the hint only where a set-aside exists
    return g_l2_reserved[dev].load(std::memory_order_relaxed) >= need ? F_KEEP_A : 0;
}

// CTAs of the root-step kernel resident at once (occupancy x SMs), per
// device and element type
template <typename T>
static int step_resident_ctas() {
    static std::atomic<int> cached[16];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) dev = 0;
    int v = cached[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        int occ = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv_step<T, OP_P_REAL, true>,
                                                          step_threads<T>(), 0) != cudaSuccess ||
            occ < 1)
            occ = 1;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            sms < 1)
            sms = 1;
        cudaGetLastError();
        v = occ * sms;
        cached[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

template <typename T, int PRE, int MINB, bool HINT>
static cudaError_t launch_direct(cudaLaunchConfig_t& cfg, int op, const StepArgs<T>& a) {
    switch (op) {
        case OP_SPMV: return cudaLaunchKernelEx(&cfg, k_spmv_direct<T, OP_SPMV, PRE, MINB, HINT>, a);
        case OP_RESID: return cudaLaunchKernelEx(&cfg, k_spmv_direct<T, OP_RESID, PRE, MINB, HINT>, a);
        case OP_PHI_REAL:
            return cudaLaunchKernelEx(&cfg, k_spmv_direct<T, OP_PHI_REAL, PRE, MINB, HINT>, a);
        case OP_PHI_PAIR2:
            return cudaLaunchKernelEx(&cfg, k_spmv_direct<T, OP_PHI_PAIR2, PRE, MINB, HINT>, a);
        case OP_P_REAL:
            return cudaLaunchKernelEx(&cfg, k_spmv_direct<T, OP_P_REAL, PRE, MINB, HINT>, a);
        case OP_P_PAIR1:
            return cudaLaunchKernelEx(&cfg, k_spmv_direct<T, OP_P_PAIR1, PRE, MINB, HINT>, a);
        case OP_P_PAIR2:
            return cudaLaunchKernelEx(&cfg, k_spmv_direct<T, OP_P_PAIR2, PRE, MINB, HINT>, a);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, bool PF>
static cudaError_t launch_op(cudaLaunchConfig_t& cfg, int op, const StepArgs<T>& a) {
    switch (op) {
        case OP_SPMV: return cudaLaunchKernelEx(&cfg, k_spmv_step<T, OP_SPMV, PF>, a);
        case OP_RESID: return cudaLaunchKernelEx(&cfg, k_spmv_step<T, OP_RESID, PF>, a);
        case OP_PHI_REAL: return cudaLaunchKernelEx(&cfg, k_spmv_step<T, OP_PHI_REAL, PF>, a);
        case OP_PHI_PAIR2: return cudaLaunchKernelEx(&cfg, k_spmv_step<T, OP_PHI_PAIR2, PF>, a);
        case OP_P_REAL: return cudaLaunchKernelEx(&cfg, k_spmv_step<T, OP_P_REAL, PF>, a);
        case OP_P_PAIR1: return cudaLaunchKernelEx(&cfg, k_spmv_step<T, OP_P_PAIR1, PF>, a);
        case OP_P_PAIR2: return cudaLaunchKernelEx(&cfg, k_spmv_step<T, OP_P_PAIR2, PF>, a);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
int32_t launch_step(int op, const StepArgs<T>& a_in, cudaStream_t s) {
    if (a_in.n <= 0) return 0;
    const int rows = step_threads<T>() * step_rpt<T>();
    const int grid = (int)(((int64_t)a_in.n + rows - 1) / rows);
    StepArgs<T> a = a_in;
    // prefetch half a resident wave ahead, unless the matrix is held in an
    // L2 set-aside (measured: the prefetches then cost more than they save).
    // 3-D 160^3 chains (FP32 / FP64) by distance in resident waves:
    // 1/4 5860 / 6121 GB/s, 1/3 6017 / 6141, 1/2 6041 / 6151, 1 5969 / 6142,
    // 3/2 5836 / 6123, 2 5218 / 5982.
    a.pf_ahead = (a.flags & F_KEEP_A) ? 0 : (step_resident_ctas<T>() + 1) / 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(step_threads<T>());
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (op < OP_SPMV || op > OP_P_PAIR2) return PPG_ERR_ARG;
    const bool small = a_in.n <= DIRECT_MAX_N;
    if (small || (a_in.flags & F_KEEP_A)) {
        // one row per thread, no staging round (small system, or matrix in L2)
        const int dgrid = (int)(((int64_t)a_in.n + SPMV_ROWS - 1) / SPMV_ROWS);
        cfg.gridDim = dim3(dgrid);
        cfg.blockDim = dim3(SPMV_ROWS);
        // matrix in L2: entries preloaded before the dependency wait -- four
        // at 32 registers (2048 threads per SM), five for the plain SpMV step
        // (still 32), five at 40 registers (1536 threads) for the second step
        // of a pair of Algorithm 1, which spills at 32 (2-D 1000^2 FP64
        // chains: staged kernel 57.3 ms; direct with four preloads 55.8 ms
        // (without the evict-last hint 56.3 ms); three for the pair step at
        // 32 registers 55.2 ms; with 128-row CTAs 54.7 ms; five for the plain
        // SpMV step 53.4 ms; five for the pair step at 40 registers 52.5 ms,
        // four there 52.8 ms)
        cudaError_t ed;
        if (small) {
            // 64-row CTAs (the residual keeps 256: one partial sum per 256
            // rows): a small system's step then spreads over 4x the SMs
            // (2-D 50^2 p(A) v 37.9 -> 32.7 us; 128 rows 35.6, 32 rows 36.8;
            // 100^2 56.1 -> 49.5 us)
            if (op != OP_RESID) {
                cfg.blockDim = dim3(DIRECT_SMALL_ROWS);
                cfg.gridDim = dim3((unsigned)(((int64_t)a_in.n + DIRECT_SMALL_ROWS - 1) /
                                              DIRECT_SMALL_ROWS));
            }
            ed = launch_direct<T, 8, 0, false>(cfg, op, a);
        } else {
            // matrix in L2: 128-row CTAs (2-D 1000^2 FP64 chains 55.22 ->
            // 54.88 ms against 256 rows; 64 rows 69.5 ms)
            if (op != OP_RESID) {
                cfg.blockDim = dim3(DIRECT_L2_ROWS);
                cfg.gridDim = dim3((unsigned)(((int64_t)a_in.n + DIRECT_L2_ROWS - 1) /
                                              DIRECT_L2_ROWS));
            }
            if (op == OP_PHI_PAIR2)   // five entries at 40 registers
                ed = launch_direct<T, 5, 6, true>(cfg, op, a);
            else if (op == OP_SPMV)   // five entries: a 5-point row whole
                ed = launch_direct<T, 5, 8, true>(cfg, op, a);
            else
                ed = launch_direct<T, 4, 8, true>(cfg, op, a);
        }
        ++g_launches;
        if (ed != cudaSuccess) {
            set_cuda_error(ed, "cudaLaunchKernelEx(k_spmv_direct)");
            return PPG_ERR_CUDA;
        }
        const int32_t rcd = check_launch("k_spmv_direct");
        return rcd < 0 ? rcd : dgrid;
    }
    const cudaError_t e =
        a.pf_ahead > 0 ? launch_op<T, true>(cfg, op, a) : launch_op<T, false>(cfg, op, a);
    ++g_launches;
    if (e != cudaSuccess) {
        set_cuda_error(e, "cudaLaunchKernelEx(k_spmv_step)");
        return PPG_ERR_CUDA;
    }
    int32_t rc = check_launch("k_spmv_step");
    return rc < 0 ? rc : grid;
}

template int32_t launch_step<double>(int, const StepArgs<double>&, cudaStream_t);
template int32_t launch_step<float>(int, const StepArgs<float>&, cudaStream_t);

// Unique bytes a step must move: the CSR (values, column indices, row
// pointers) once, and each distinct length-n vector it reads or writes once.
double step_bytes(int op, int flags, int64_t n, int64_t nnz, int elem) {
    double M = (double)nnz * (elem + 4) + 4.0 * (double)(n + 1);
    int vec = 0;
    switch (op) {
        case OP_SPMV: vec = 2; break;
        case OP_RESID: vec = 3; break;
        case OP_PHI_REAL: vec = (flags & F_FINAL) ? 3 : 2; break;
        case OP_PHI_PAIR2: vec = (flags & F_FINAL) ? 4 : 3; break;
        case OP_P_REAL:
            vec = 2 + ((flags & F_PZERO) ? 0 : 1) + ((flags & F_FINAL) ? 0 : 1);
            break;
        case OP_P_PAIR1:
            vec = 2 + ((flags & F_PZERO) ? 0 : 1) + ((flags & F_NO_O1) ? 0 : 1);
            break;
        case OP_P_PAIR2: vec = (flags & F_FINAL) ? 4 : 3; break;
        default: break;
    }
    return M + (double)vec * (double)elem * (double)n;
}

}  // namespace ppg
