// Orthogonalisation (CGS2) and the small dense steps of GMRES: Givens
// least squares (Section 3.2 shortcut residual), back substitution, the
// solution update V y, norms and scaling.
//
// The basis V is column-major with leading dimension ldv (>= n, padded so
// each column starts on a 512-byte boundary).  Classical Gram-Schmidt
// applied twice runs as four streaming passes over the active columns:
//   h1 = V^T w ;  w -= V h1 ;  h2 = V^T w ;  w -= V h2 (and ||w||^2)
// Each pass spends exactly one FP64 fused multiply-add per element of V --
// on GB300 the FP64 pipe (about two operations per clock per SM), not HBM,
// is the tighter bound for this work -- and keeps many independent loads in
// flight per thread.  The dot pass accumulates eight columns per thread in
// registers, reduces them across the warp with an exchange tree of nine
// shuffles for all eight, and the last CTA to finish sums the per-CTA
// partials in a fixed order (deterministic; the counter resets itself, no
// waiting, no extra launch).
#include <atomic>

#include "ppg_common.cuh"

namespace ppg {

constexpr int ORTHO_THREADS = 256;
constexpr int ORTHO_WARPS = ORTHO_THREADS / 32;
constexpr int DOT_CH = 8;                 // columns per register chunk
constexpr int PART_STRIDE = ORTHO_MAXC + 2;
// threads per CTA of the two streaming CGS2 passes (k_mdot, k_gemv_sub),
// their minimum CTAs per SM, and the most row blocks they launch (one wave)
constexpr int CGS_THREADS = 256;
constexpr int CGS_WARPS = CGS_THREADS / 32;
constexpr int CGS_DOT_MINB = 4 * 256 / CGS_THREADS;
constexpr int CGS_SUB_MINB = 5 * 256 / CGS_THREADS;
inline int cgs_max_blocks() { return grid_cap(8 * 256 / CGS_THREADS); }

int ortho_grid(int32_t n) {
    const int per = ORTHO_THREADS * 8;   // at least ~8 rows per thread
    return max(1, min((n + per - 1) / per, grid_cap(2)));
}

// partial sums of the CGS2 passes: their grids have at most cgs_max_blocks()
// row blocks (the norm kernels at most `grid`)
size_t ortho_part_doubles(int grid) {
    return (size_t)max(grid, max(grid_cap(8), cgs_max_blocks())) * PART_STRIDE;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

// Sum each of v[0..7] over the 32 lanes.  Afterwards lane l with (l & 3) == 0
// holds the total of value l >> 2 in v[0].
__device__ __forceinline__ void warp_reduce8(double v[8], int lane) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool hi = lane & 16;
        const double send = hi ? v[i] : v[i + 4];
        const double keep = hi ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool hi = lane & 8;
        const double send = hi ? v[i] : v[i + 2];
        const double keep = hi ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    {
        const bool hi = lane & 4;
        const double send = hi ? v[0] : v[1];
        const double keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Reduce part[b * PART_STRIDE + c] over b < nblocks for c < nvals, in block
// order, into out[c].  Called by every thread of the last CTA.
__device__ void final_reduce(const double* part, int nblocks, int nvals, double* out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = warp; c < nvals; c += (int)(blockDim.x >> 5)) {
        double s = 0.0;
        for (int b = lane; b < nblocks; b += 32) s += __ldcg(part + (size_t)b * PART_STRIDE + c);
        s = warp_sum(s);
        if (lane == 0) out[c] = s;
    }
}

__device__ __forceinline__ bool last_block_done(unsigned* counter) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    return am_last;
}

// acc[q] += sum over this thread's rows of col[q][r] w[r], q < NQ: two rows
// per trip, so 2 (NQ + 1) loads are in flight.  NQ is a compile-time width:
// a predicated-off FP64 FMA still occupies the FP64 pipe on GB300, so the
// last, narrower chunk of columns must not issue FMAs for missing columns.
template <int NQ, bool VEC2>
__device__ __forceinline__ void dot_rows(const double* const* col, const double* __restrict__ w,
                                         int64_t r, int64_t stride, int64_t n, double* acc) {
    if constexpr (VEC2) {
        // rows 2p and 2p+1 with one 16-byte load per column (half the load
        // instructions of two 8-byte loads); an odd last row goes to the one
        // thread whose pair index stops at n / 2
        const int64_t np = n >> 1;
        int64_t p = r;
        for (; p < np; p += stride) {
            const double2 w2 = __ldg(reinterpret_cast<const double2*>(w) + p);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const double2 a = __ldcs(reinterpret_cast<const double2*>(col[q]) + p);
                acc[q] = fma(a.y, w2.y, fma(a.x, w2.x, acc[q]));
            }
        }
        if ((n & 1) && p == np) {
            const double w0 = w[n - 1];
#pragma unroll
            for (int q = 0; q < NQ; ++q) acc[q] = fma(__ldcs(col[q] + n - 1), w0, acc[q]);
        }
    } else {
        // acc[q] += sum over this thread's rows of col[q][r] w[r], two rows
        // per trip, so 2 (NQ + 1) loads are in flight
        for (; r + stride < n; r += 2 * stride) {
            const double w0 = w[r], w1 = w[r + stride];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const double a0 = __ldcs(col[q] + r), a1 = __ldcs(col[q] + r + stride);
                acc[q] = fma(a1, w1, fma(a0, w0, acc[q]));
            }
        }
        if (r < n) {
            const double w0 = w[r];
#pragma unroll
            for (int q = 0; q < NQ; ++q) acc[q] = fma(__ldcs(col[q] + r), w0, acc[q]);
        }
    }
}

// hout[c] = sum_r V[c][r] w[r] for c < ncol, and hout[ncol] = w.w when
// with_self.  Grid: x = row blocks (grid-stride), y = chunks of eight
// columns, so every column chunk streams in parallel.
template <bool VEC2>
__global__ void __launch_bounds__(CGS_THREADS, CGS_DOT_MINB)
k_mdot(const double* __restrict__ V, int64_t ldv, int ncol, const double* __restrict__ w,
       int32_t n, int with_self, double* part, unsigned* counter, double* hout) {
    __shared__ double sred[CGS_WARPS][DOT_CH];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nvals = ncol + (with_self ? 1 : 0);
    // gridDim.y = ceil(nvals / 8) chunks of near-equal width (at most 8), so
    // no CTA of the single wave is left with a narrow remainder
    const int c0 = (int)(blockIdx.y * (unsigned)nvals / gridDim.y);
    const int nq = (int)((blockIdx.y + 1) * (unsigned)nvals / gridDim.y) - c0;
    const double* col[DOT_CH];
#pragma unroll
    for (int q = 0; q < DOT_CH; ++q) {
        const int c = c0 + q;
        col[q] = (c < ncol) ? V + c * ldv : w;
    }
    double acc[DOT_CH];
#pragma unroll
    for (int q = 0; q < DOT_CH; ++q) acc[q] = 0.0;
    PPG_PDL_TRIGGER();
    PPG_PDL_WAIT();
    const int64_t stride = (int64_t)gridDim.x * CGS_THREADS;
    const int64_t r = (int64_t)blockIdx.x * CGS_THREADS + tid;
    switch (nq) {
        case 8: dot_rows<8, VEC2>(col, w, r, stride, n, acc); break;
        case 7: dot_rows<7, VEC2>(col, w, r, stride, n, acc); break;
        case 6: dot_rows<6, VEC2>(col, w, r, stride, n, acc); break;
        case 5: dot_rows<5, VEC2>(col, w, r, stride, n, acc); break;
        case 4: dot_rows<4, VEC2>(col, w, r, stride, n, acc); break;
        case 3: dot_rows<3, VEC2>(col, w, r, stride, n, acc); break;
        case 2: dot_rows<2, VEC2>(col, w, r, stride, n, acc); break;
        default: dot_rows<1, VEC2>(col, w, r, stride, n, acc); break;
    }
    warp_reduce8(acc, lane);
    if ((lane & 3) == 0) sred[warp][lane >> 2] = acc[0];
    __syncthreads();
    if (tid < nq) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < CGS_WARPS; ++k) t += sred[k][tid];
        part[(size_t)blockIdx.x * PART_STRIDE + c0 + tid] = t;
    }
    // the last CTA of the whole grid sums the partials of every column
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (tid == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x * gridDim.y - 1);
    __syncthreads();
    if (am_last) {
        __threadfence();
        final_reduce(part, gridDim.x, nvals, hout);
        if (tid == 0) *counter = 0u;
    }
}

// w[r] -= sum_c V[c][r] h[c]; with_norm: nout[0] = ||w||^2 afterwards
template <bool VEC2>
__global__ void __launch_bounds__(CGS_THREADS, CGS_SUB_MINB)
k_gemv_sub(const double* __restrict__ V, int64_t ldv, int ncol, double* w, int32_t n,
           const double* __restrict__ h, int with_norm, double* part, unsigned* counter,
           double* nout) {
    __shared__ double sh[ORTHO_MAXC];
    __shared__ double sred[CGS_WARPS];
    const int tid = threadIdx.x;
    PPG_PDL_TRIGGER();
    PPG_PDL_WAIT();
    for (int c = tid; c < ncol; c += CGS_THREADS) sh[c] = h[c];
    __syncthreads();
    double nacc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * CGS_THREADS;
    int64_t r = (int64_t)blockIdx.x * CGS_THREADS + tid;
    if constexpr (VEC2) {
        // rows 2p and 2p+1: one 16-byte load per column, two FMA chains,
        // exactly one FMA per element of V; an odd last row goes to the one
        // thread whose pair index stops at n / 2
        const int64_t np = (int64_t)n >> 1;
        int64_t p = r;
        for (; p < np; p += stride) {
            double s0 = 0.0, s1 = 0.0;
            for (int c = 0; c < ncol; ++c) {
                const double hc = sh[c];
                const double2 v = __ldcs(reinterpret_cast<const double2*>(V + c * ldv) + p);
                s0 = fma(v.x, hc, s0);
                s1 = fma(v.y, hc, s1);
            }
            double2 w2 = reinterpret_cast<double2*>(w)[p];
            w2.x -= s0;
            w2.y -= s1;
            reinterpret_cast<double2*>(w)[p] = w2;
            nacc = fma(w2.y, w2.y, fma(w2.x, w2.x, nacc));
        }
        // the odd last row: taken below by the one thread whose pair index
        // stopped at n / 2
        r = ((n & 1) && p == np) ? (int64_t)n - 1 : (int64_t)n;
    } else {
        // two rows per trip: two independent FMA chains, 2 loads per column
        // in flight, exactly one FMA per element of V
        for (; r + stride < n; r += 2 * stride) {
            double s0 = 0.0, s1 = 0.0;
            for (int c = 0; c < ncol; ++c) {
                const double hc = sh[c];
                s0 = fma(__ldcs(V + c * ldv + r), hc, s0);
                s1 = fma(__ldcs(V + c * ldv + r + stride), hc, s1);
            }
            const double w0 = w[r] - s0, w1 = w[r + stride] - s1;
            w[r] = w0;
            w[r + stride] = w1;
            nacc = fma(w1, w1, fma(w0, w0, nacc));
        }
    }
    if (r < n) {
        double s0 = 0.0;
        for (int c = 0; c < ncol; ++c) s0 = fma(__ldcs(V + c * ldv + r), sh[c], s0);
        const double w0 = w[r] - s0;
        w[r] = w0;
        nacc = fma(w0, w0, nacc);
    }
    if (!with_norm) return;
    nacc = warp_sum(nacc);
    if ((tid & 31) == 0) sred[tid >> 5] = nacc;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int k = 0; k < CGS_WARPS; ++k) t += sred[k];
        part[(size_t)blockIdx.x * PART_STRIDE] = t;
    }
    if (last_block_done(counter)) {
        __threadfence();
        final_reduce(part, gridDim.x, 1, nout);
        if (tid == 0) *counter = 0u;
    }
}

// ---------------------------------------------------------------------------
// CGS2 passes 2 and 3 in one pass over V:  w -= V h1, then h2 = V^T w of the
// updated w.  The update of a row needs only that row of V, so a tile of
// rows is read from HBM once and serves both products: 3/4 of the unfused
// passes' bytes, the same FP64 multiply-adds.
//
// Tiles of SD_R rows x ncol columns move from HBM to shared memory with one
// bulk copy per column (the TMA engine; column c of the tile is one
// contiguous 1 KB range of the column-major basis), double buffered on two
// mbarriers.  Each thread then takes a register block of the tile -- warp k
// owns a contiguous run of at most SD_CPW columns, lane l the rows 2l, 2l+1,
// 64+2l, 65+2l -- with one 16-byte shared load per two elements, and uses
// it twice: phase 1 sums V[r, c] h1[c] over the warp's columns into
// per-warp row partials, which are added in warp order to give
// w' = w - V h1; phase 2 adds V[r, c] w'[r] into per-column accumulators
// that persist across the CTA's tiles.  So every element costs two FP64
// multiply-adds and half a shared load: on GB300, where the FP64 pipe
// issues at half the instruction rate, the multiply-adds set the pace.
// Per-CTA partial sums are reduced by the last CTA in a fixed order
// (deterministic).
//
// Every wait on an mbarrier is bounded; a CTA whose copies do not arrive
// sets *err, waits (bounded) for the copies it issued, and returns.
// ---------------------------------------------------------------------------

constexpr int SD_R = 128;                 // rows per tile
constexpr int SD_MAXC = 56;               // columns (at most 7 per warp)
constexpr int SD_CPW = SD_MAXC / ORTHO_WARPS;
constexpr uint32_t SD_SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for phase `parity` of the mbarrier at `bar`
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    for (uint32_t it = 0; it < SD_SPIN_LIMIT; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Shared-memory layout of k_sub_dot besides the staged tiles.
struct SubDotShared {
    double spart[ORTHO_WARPS][SD_R];
    double ws[SD_R];
    uint64_t bar[2];
};

// The tile loop of k_sub_dot for a warp owning NC columns (a compile-time
// count: on GB300 a predicated or discarded FP64 multiply-add still takes
// its FP64 pipe slot, so missing columns must not appear in the code).
// Warps of one CTA may run different instantiations; they meet at the same
// barriers.
template <int NC>
__device__ __forceinline__ void sub_dot_tiles(const double* __restrict__ V, int64_t ldv, int ncol,
                                              double* w, int32_t n, const double* __restrict__ h1,
                                              double* part, unsigned* counter, double* hout,
                                              unsigned* err, double* sd_stage,
                                              SubDotShared& sm, int c0) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t stage_elems = (int64_t)ncol * SD_R;
    const int ntiles = (int)(((int64_t)n + SD_R - 1) / SD_R);
    double hreg[NC > 0 ? NC : 1];
#pragma unroll
    for (int k = 0; k < NC; ++k) hreg[k] = h1[c0 + k];

    // thread 0: tile t into stage st (rows up to the padded column length,
    // a multiple of 64 rows, so every copy is a whole number of 16 bytes)
    auto issue = [&](int t, int st) {
        const int64_t r0 = (int64_t)t * SD_R;
        const int64_t rows = min((int64_t)SD_R, ldv - r0);
        const uint32_t bytes = (uint32_t)(rows * 8);
        const uint32_t b = smem_u32(&sm.bar[st]);
        double* dst = sd_stage + st * stage_elems;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
                     "r"(bytes * (uint32_t)ncol)
                     : "memory");
        for (int c = 0; c < ncol; ++c) {
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                ::"r"(smem_u32(dst + c * SD_R)), "l"(V + c * ldv + r0), "r"(bytes), "r"(b)
                : "memory");
        }
    };
    const int first = blockIdx.x;
    const int step = gridDim.x;
    if (tid == 0) {
        if (first < ntiles) issue(first, 0);
        if (first + step < ntiles) issue(first + step, 1);
    }

    double acc[NC > 0 ? NC : 1];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = 0.0;
    int k_local = 0;
    bool ok = true;
    for (int t = first; t < ntiles; t += step, ++k_local) {
        const int st = k_local & 1;
        const int64_t r0 = (int64_t)t * SD_R;
        // the combining threads fetch their two rows of w early
        double2 wv = make_double2(0.0, 0.0);
        const int64_t gw = r0 + 2 * tid;
        if (tid < SD_R / 2) {
            if (gw + 1 < n) {
                wv = *reinterpret_cast<const double2*>(w + gw);
            } else if (gw < n) {
                wv.x = w[gw];
            }
        }
        const bool mine =
            mbar_wait_bounded(smem_u32(&sm.bar[st]), (uint32_t)((k_local >> 1) & 1));
        if (!__syncthreads_and(mine)) {
            ok = false;
            break;
        }
        const double* S = sd_stage + st * stage_elems;
        // this thread's register block; rows at or past n hold the basis's
        // padding (never written, possibly not finite) and become zeros
        double2 va[NC > 0 ? NC : 1], vb[NC > 0 ? NC : 1];
        const bool full = r0 + SD_R <= n;
        const int64_t ra = r0 + 2 * lane, rb = r0 + 64 + 2 * lane;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            va[k] = *reinterpret_cast<const double2*>(S + (c0 + k) * SD_R + 2 * lane);
            vb[k] = *reinterpret_cast<const double2*>(S + (c0 + k) * SD_R + 64 + 2 * lane);
            if (!full) {
                va[k].x = ra < n ? va[k].x : 0.0;
                va[k].y = ra + 1 < n ? va[k].y : 0.0;
                vb[k].x = rb < n ? vb[k].x : 0.0;
                vb[k].y = rb + 1 < n ? vb[k].y : 0.0;
            }
        }
        // phase 1: row partials of V h1 over this warp's columns
        {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                s0 = fma(va[k].x, hreg[k], s0);
                s1 = fma(va[k].y, hreg[k], s1);
                s2 = fma(vb[k].x, hreg[k], s2);
                s3 = fma(vb[k].y, hreg[k], s3);
            }
            *reinterpret_cast<double2*>(&sm.spart[warp][2 * lane]) = make_double2(s0, s1);
            *reinterpret_cast<double2*>(&sm.spart[warp][64 + 2 * lane]) = make_double2(s2, s3);
        }
        __syncthreads();   // the stage is in registers; the partials are complete
        if (tid == 0 && t + 2 * step < ntiles) {
            // order this CTA's reads of the stage before the bulk copy that
            // overwrites it
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(t + 2 * step, st);
        }
        if (tid < SD_R / 2) {
            const int r = 2 * tid;
            double sa = 0.0, sb = 0.0;
#pragma unroll
            for (int g = 0; g < ORTHO_WARPS; ++g) {
                sa += sm.spart[g][r];
                sb += sm.spart[g][r + 1];
            }
            double2 o;
            o.x = gw < n ? wv.x - sa : 0.0;
            o.y = gw + 1 < n ? wv.y - sb : 0.0;
            *reinterpret_cast<double2*>(sm.ws + r) = o;
            if (gw + 1 < n) {
                *reinterpret_cast<double2*>(w + gw) = o;
            } else if (gw < n) {
                w[gw] = o.x;
            }
        }
        __syncthreads();
        // phase 2: column partials of V^T w' over this lane's four rows
        {
            const double2 wa = *reinterpret_cast<const double2*>(sm.ws + 2 * lane);
            const double2 wb = *reinterpret_cast<const double2*>(sm.ws + 64 + 2 * lane);
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                acc[k] = fma(va[k].x, wa.x, acc[k]);
                acc[k] = fma(va[k].y, wa.y, acc[k]);
                acc[k] = fma(vb[k].x, wb.x, acc[k]);
                acc[k] = fma(vb[k].y, wb.y, acc[k]);
            }
        }
    }
    if (!ok) {
        // the copies did not arrive: flag it, give the copies this CTA issued
        // a bounded chance to land, and leave without touching the results
        if (tid == 0) {
            atomicExch(err, 1u);
            for (int j = 0; j < 2; ++j) {
                const int kk = k_local + j;   // outstanding tiles k_local, k_local + 1
                if (first + kk * step < ntiles)
                    mbar_wait_bounded(smem_u32(&sm.bar[kk & 1]), (uint32_t)((kk >> 1) & 1));
            }
        }
        return;
    }
    // per-CTA partial sums of each column over this CTA's rows
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) part[(size_t)blockIdx.x * PART_STRIDE + c0 + k] = v;
    }
    if (last_block_done(counter)) {
        __threadfence();
        final_reduce(part, gridDim.x, ncol, hout);
        if (tid == 0) *counter = 0u;
    }
}

__global__ void __launch_bounds__(ORTHO_THREADS, 2)
k_sub_dot(const double* __restrict__ V, int64_t ldv, int ncol, double* w, int32_t n,
          const double* __restrict__ h1, double* part, unsigned* counter, double* hout,
          unsigned* err) {
    extern __shared__ __align__(128) double sd_stage[];   // 2 x ncol x SD_R
    __shared__ __align__(16) SubDotShared sm;
    const int tid = threadIdx.x, warp = tid >> 5;
    // this warp's columns [c0, c0 + nc), near-equal runs
    const int c0 = warp * ncol / ORTHO_WARPS;
    const int nc = (warp + 1) * ncol / ORTHO_WARPS - c0;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    PPG_PDL_TRIGGER();
    PPG_PDL_WAIT();   // h1 and w come from the kernels before this one
    __syncthreads();
#define PPG_SD_CASE(K)                                                                      \
    case K:                                                                                 \
        sub_dot_tiles<K>(V, ldv, ncol, w, n, h1, part, counter, hout, err, sd_stage, sm, c0); \
        break;
    switch (nc) {   // uniform over the warp
        PPG_SD_CASE(0)
        PPG_SD_CASE(1)
        PPG_SD_CASE(2)
        PPG_SD_CASE(3)
        PPG_SD_CASE(4)
        PPG_SD_CASE(5)
        PPG_SD_CASE(6)
        default: sub_dot_tiles<7>(V, ldv, ncol, w, n, h1, part, counter, hout, err, sd_stage, sm, c0);
    }
#undef PPG_SD_CASE
}

// CTAs of a kernel resident at once on the current device (occupancy x
// SMs), cached per device and kernel slot
template <typename K>
static int resident_ctas(K kernel, int slot, int threads) {
    static std::atomic<int> cached[16][4];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) dev = 0;
    int v = cached[dev][slot].load(std::memory_order_relaxed);
    if (v == 0) {
        int occ = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) !=
                cudaSuccess || occ < 1)
            occ = 4;
        sms = device_sm_count();
        v = occ * sms;
        cached[dev][slot].store(v, std::memory_order_relaxed);
    }
    return v;
}
// 16-byte (double2) loads when V, its column stride and w allow them
static bool vec2_ok(const double* V, int64_t ldv, const double* w) {
    return (((uintptr_t)V | (uintptr_t)w) & 15) == 0 && (ldv & 1) == 0;
}

int32_t launch_cgs_dot(const double* V, int64_t ldv, int ncol, const double* w, int32_t n,
                       bool with_self, double* h_out, const OrthoWs& ws, cudaStream_t s) {
    if (ncol < 1 || ncol + 1 > ORTHO_MAXC + 2) return PPG_ERR_ARG;
    const int nvals = ncol + (with_self ? 1 : 0);
    const int nch = (nvals + DOT_CH - 1) / DOT_CH;
    // row blocks x column chunks = one full wave of resident CTAs (at least
    // two rows per thread; the partial-sum buffer holds cgs_max_blocks() row
    // blocks)
    const bool v2 = vec2_ok(V, ldv, w);
    const int slots = v2 ? resident_ctas(k_mdot<true>, 0, CGS_THREADS)
                         : resident_ctas(k_mdot<false>, 1, CGS_THREADS);
    const int gx = max(1, min(min(slots / nch, (n + 2 * CGS_THREADS - 1) / (2 * CGS_THREADS)),
                              cgs_max_blocks()));
    const dim3 grid(gx, nch);
    const cudaError_t e =
        v2 ? launch_pdl(k_mdot<true>, grid, dim3(CGS_THREADS), 0, s, V, ldv, ncol, w, n,
                        with_self ? 1 : 0, ws.part, ws.counter, h_out)
           : launch_pdl(k_mdot<false>, grid, dim3(CGS_THREADS), 0, s, V, ldv, ncol, w, n,
                        with_self ? 1 : 0, ws.part, ws.counter, h_out);
    ++g_launches;
    if (e != cudaSuccess) { set_cuda_error(e, "launch k_mdot"); return PPG_ERR_CUDA; }
    return check_launch("k_mdot");
}

int32_t launch_cgs_update(const double* V, int64_t ldv, int ncol, double* w, int32_t n,
                          const double* hin, bool with_norm, double* nrm_out,
                          const OrthoWs& ws, cudaStream_t s) {
    if (ncol < 1 || ncol > ORTHO_MAXC) return PPG_ERR_ARG;
    // one wave of resident CTAs, at least two rows per thread, at most the
    // cgs_max_blocks() row blocks the partial-sum buffer holds
    const bool v2 = vec2_ok(V, ldv, w);
    const int slots = v2 ? resident_ctas(k_gemv_sub<true>, 2, CGS_THREADS)
                         : resident_ctas(k_gemv_sub<false>, 3, CGS_THREADS);
    const int grid = max(1, min(min(slots, (n + 2 * CGS_THREADS - 1) / (2 * CGS_THREADS)),
                                cgs_max_blocks()));
    const cudaError_t e =
        v2 ? launch_pdl(k_gemv_sub<true>, dim3(grid), dim3(CGS_THREADS), 0, s, V, ldv, ncol, w,
                        n, hin, with_norm ? 1 : 0, ws.part, ws.counter + 1, nrm_out)
           : launch_pdl(k_gemv_sub<false>, dim3(grid), dim3(CGS_THREADS), 0, s, V, ldv, ncol,
                        w, n, hin, with_norm ? 1 : 0, ws.part, ws.counter + 1, nrm_out);
    ++g_launches;
    if (e != cudaSuccess) { set_cuda_error(e, "launch k_gemv_sub"); return PPG_ERR_CUDA; }
    return check_launch("k_gemv_sub");
}

// the fused pass applies when V's columns and w are 16-byte aligned and
// padded to ldv rows (a multiple of 64: every tile copy is whole 16-byte
// granules), w is a column of the same padded basis, and ncol <= SD_MAXC
bool cgs_fused_ok(const double* V, int64_t ldv, int ncol, const double* w) {
    return ncol >= 1 && ncol <= SD_MAXC && (ldv % 64) == 0 &&
           (((uintptr_t)V | (uintptr_t)w) & 15) == 0;
}

static size_t sub_dot_smem(int ncol) { return (size_t)2 * ncol * SD_R * sizeof(double); }

// resident CTAs of k_sub_dot for a column count (dynamic shared memory
// depends on it), cached per device
static int sub_dot_resident(int ncol) {
    static std::atomic<int> cached[16][SD_MAXC + 1];
    static std::atomic<int> attr_set[16];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) dev = 0;
    if (!attr_set[dev].load(std::memory_order_relaxed)) {
        cudaFuncSetAttribute(k_sub_dot, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sub_dot_smem(SD_MAXC));
        attr_set[dev].store(1, std::memory_order_relaxed);
    }
    int v = cached[dev][ncol].load(std::memory_order_relaxed);
    if (v == 0) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sub_dot, ORTHO_THREADS,
                                                          sub_dot_smem(ncol)) != cudaSuccess ||
            occ < 1) {
            cudaGetLastError();
            occ = 1;
        }
        v = occ * device_sm_count();
        cached[dev][ncol].store(v, std::memory_order_relaxed);
    }
    return v;
}

int32_t launch_cgs_sub_dot(const double* V, int64_t ldv, int ncol, double* w, int32_t n,
                           const double* h1, double* h2_out, const OrthoWs& ws,
                           cudaStream_t s) {
    if (!cgs_fused_ok(V, ldv, ncol, w) || n < 1 || ldv < n) return PPG_ERR_ARG;
    const int ntiles = (int)(((int64_t)n + SD_R - 1) / SD_R);
    // one wave of resident CTAs, at most the grid_cap(8) row blocks the
    // partial-sum buffer holds
    const int grid = max(1, min(min(sub_dot_resident(ncol), ntiles), grid_cap(8)));
    const cudaError_t e = launch_pdl(k_sub_dot, dim3(grid), dim3(ORTHO_THREADS),
                                     sub_dot_smem(ncol), s, V, ldv, ncol, w, n, h1, ws.part,
                                     ws.counter + 2, h2_out, ws.counter + 3);
    ++g_launches;
    if (e != cudaSuccess) { set_cuda_error(e, "launch k_sub_dot"); return PPG_ERR_CUDA; }
    return check_launch("k_sub_dot");
}

// ---------------------------------------------------------------------------
// Hessenberg column, Givens rotation, shortcut residual (one thread)
// ---------------------------------------------------------------------------

__global__ void k_finish_column(GmresState st, int ldh, int j, const double* h1,
                                const double* h2, const double* nrm, int givens,
                                double bnorm, double brtol) {
    // one warp stages the column and the rotations in shared memory, then
    // one thread applies the j earlier rotations and makes the new one
    __shared__ double col[ORTHO_MAXC + 1];
    __shared__ double scs[ORTHO_MAXC], ssn[ORTHO_MAXC];
    const int lane = threadIdx.x;
    PPG_PDL_TRIGGER();
    PPG_PDL_WAIT();
    for (int i = lane; i <= j; i += 32) col[i] = h1[i] + h2[i];
    if (givens)
        for (int i = lane; i < j; i += 32) {
            scs[i] = st.cs[i];
            ssn[i] = st.sn[i];
        }
    const double hn = sqrt(fmax(nrm[0], 0.0));
    if (lane == 0) col[j + 1] = hn;
    __syncwarp();
    if (st.Hraw)
        for (int i = lane; i <= j + 1; i += 32) st.Hraw[(size_t)j * ldh + i] = col[i];
    __syncwarp();
    if (lane != 0) return;
    double* sc = st.scal;
    bool brk;
    if (brtol > 0.0) {
        const double w0 = sqrt(fmax(h1[j + 1], 0.0));   // ||A v_j|| from the first dot pass
        brk = !(hn > brtol * w0);
    } else {
        brk = !(hn > 0.0);
    }
    if (brk && sc[5] == 0.0) {
        sc[5] = 1.0;
        sc[6] = (double)j;
    }
    if (brk && st.Hraw) st.Hraw[(size_t)j * ldh + j + 1] = 0.0;
    sc[1] = hn;
    sc[2] = (hn > 0.0 && !brk) ? 1.0 / hn : 0.0;
    if (givens) {
        double ci = col[0];
        for (int i = 0; i < j; ++i) {
            const double nxt = col[i + 1];
            const double t = scs[i] * ci + ssn[i] * nxt;
            ci = -ssn[i] * ci + scs[i] * nxt;
            col[i] = t;
        }
        col[j] = ci;
        const double a = col[j], b = col[j + 1];
        const double r = hypot(a, b);
        double c = 1.0, s = 0.0;
        if (r != 0.0) { c = a / r; s = b / r; }
        st.cs[j] = c;
        st.sn[j] = s;
        col[j] = r;
        for (int i = 0; i <= j; ++i) st.R[(size_t)j * ldh + i] = col[i];
        const double gj = st.g[j];
        st.g[j + 1] = -s * gj;
        st.g[j] = c * gj;
        sc[0] = fabs(st.g[j + 1]) / bnorm;
    }
}

int32_t launch_finish_column(const GmresState& st, int ldh, int j, const double* h1,
                             const double* h2, const double* nrm, bool givens,
                             double bnorm, double brtol, cudaStream_t s) {
    if (j + 1 > ORTHO_MAXC) return PPG_ERR_ARG;
    const cudaError_t e = launch_pdl(k_finish_column, dim3(1), dim3(32), 0, s, st, ldh, j, h1,
                                     h2, nrm, givens ? 1 : 0, bnorm, brtol);
    ++g_launches;
    if (e != cudaSuccess) { set_cuda_error(e, "launch k_finish_column"); return PPG_ERR_CUDA; }
    return check_launch("k_finish_column");
}

// y = R^{-1} g (k x k upper triangular; R[i][c] at R[c * ldh + i]).  The
// CTA stages R in shared memory (k <= BS_MAXK), then one warp solves from
// the bottom row up: for row i the lanes share the sum over the solved
// entries c > i, lane 0 divides.  Larger k reads R from global memory.
constexpr int BS_MAXK = 64;

__global__ void __launch_bounds__(256) k_backsolve(GmresState st, int ldh, int k) {
    __shared__ double sR[BS_MAXK * BS_MAXK];
    __shared__ double sy[ORTHO_MAXC];
    const int tid = threadIdx.x, lane = tid & 31;
    const bool staged = k <= BS_MAXK;
    if (staged)
        for (int e = tid; e < k * k; e += blockDim.x) {
            const int c = e / k, i = e - c * k;
            if (i <= c) sR[c * BS_MAXK + i] = st.R[(size_t)c * ldh + i];
        }
    __syncthreads();
    if (tid >= 32) return;
    for (int i = k - 1; i >= 0; --i) {
        double part = 0.0;
        for (int c = i + 1 + lane; c < k; c += 32)
            part = fma(staged ? sR[c * BS_MAXK + i] : st.R[(size_t)c * ldh + i], sy[c], part);
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        if (lane == 0)
            sy[i] = (st.g[i] - part) / (staged ? sR[i * BS_MAXK + i] : st.R[(size_t)i * ldh + i]);
        __syncwarp();
    }
    for (int i = lane; i < k; i += 32) st.y[i] = sy[i];
}

int32_t launch_backsolve(const GmresState& st, int ldh, int k, cudaStream_t s) {
    k_backsolve<<<1, 256, 0, s>>>(st, ldh, k);
    ++g_launches;
    return check_launch("k_backsolve");
}

// out = (accumulate ? out : 0) + V[:, :k] y
template <typename TV>
__global__ void k_gemv_acc(const TV* __restrict__ V, int64_t ldv, int k,
                           const double* __restrict__ y, double* out, int32_t n,
                           int accumulate) {
    __shared__ double sy[ORTHO_MAXC];
    for (int c = threadIdx.x; c < k; c += blockDim.x) sy[c] = y[c];
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        double s = accumulate ? out[r] : 0.0;
        for (int c = 0; c < k; ++c) s += (double)__ldcs(V + c * ldv + r) * sy[c];
        out[r] = s;
    }
}

template <typename TV>
int32_t launch_gemv_acc(const TV* V, int64_t ldv, int k, const double* y, double* out,
                        int32_t n, bool accumulate, cudaStream_t s) {
    if (k < 0 || k > ORTHO_MAXC) return PPG_ERR_ARG;
    const int grid = max(1, min((n + 255) / 256, grid_cap(8)));
    k_gemv_acc<TV><<<grid, 256, 0, s>>>(V, ldv, k, y, out, n, accumulate ? 1 : 0);
    ++g_launches;
    return check_launch("k_gemv_acc");
}
template int32_t launch_gemv_acc<double>(const double*, int64_t, int, const double*,
                                         double*, int32_t, bool, cudaStream_t);
template int32_t launch_gemv_acc<float>(const float*, int64_t, int, const double*,
                                        double*, int32_t, bool, cudaStream_t);

// y = x * scal[2]   (x may equal y)
__global__ void k_scale(const double* x, double* y, int32_t n, const double* sp) {
    PPG_PDL_TRIGGER();
    PPG_PDL_WAIT();
    const double a = *sp;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        y[r] = x[r] * a;
}

int32_t launch_scale(const double* x, double* y, int32_t n, const double* sp,
                     cudaStream_t s) {
    const int grid = max(1, min((n + 255) / 256, grid_cap(8)));
    const cudaError_t e = launch_pdl(k_scale, dim3(grid), dim3(256), 0, s, x, y, n, sp);
    ++g_launches;
    if (e != cudaSuccess) { set_cuda_error(e, "launch k_scale"); return PPG_ERR_CUDA; }
    return check_launch("k_scale");
}

// partial sums of x.x (or (a-b).(a-b)) per CTA
template <bool DIFF>
__global__ void k_norm2_part(const double* a, const double* b, int32_t n, double* part) {
    __shared__ double sred[8];
    double s = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const double v = DIFF ? a[r] - b[r] : a[r];
        s += v * v;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sred[w];
        part[blockIdx.x] = t;
    }
}

int32_t launch_norm2_part(const double* x, int32_t n, double* part, cudaStream_t s,
                          int* nparts) {
    const int grid = max(1, min((n + 255) / 256, grid_cap(4)));
    k_norm2_part<false><<<grid, 256, 0, s>>>(x, nullptr, n, part);
    ++g_launches;
    *nparts = grid;
    return check_launch("k_norm2_part");
}

int32_t launch_diff_norm2_part(const double* a, const double* b, int32_t n, double* part,
                               cudaStream_t s, int* nparts) {
    const int grid = max(1, min((n + 255) / 256, grid_cap(4)));
    k_norm2_part<true><<<grid, 256, 0, s>>>(a, b, n, part);
    ++g_launches;
    *nparts = grid;
    return check_launch("k_norm2_part");
}

// beta = sqrt(sum part); scal[3] = beta, scal[4] = 1/beta; g0 = beta
__global__ void k_reduce_norm(const double* part, int nparts, double* scal, double* g0) {
    __shared__ double sred[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sred[w];
        const double beta = sqrt(t);
        scal[3] = beta;
        scal[4] = (beta > 0.0) ? 1.0 / beta : 0.0;
        if (g0) *g0 = beta;
    }
}

int32_t launch_reduce_norm(const double* part, int nparts, double* scal, double* g0,
                           cudaStream_t s) {
    k_reduce_norm<<<1, 1024, 0, s>>>(part, nparts, scal, g0);
    ++g_launches;
    return check_launch("k_reduce_norm");
}

__global__ void k_cast_f64_f32(const double* x, float* y, int32_t n) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        y[r] = (float)x[r];
}
__global__ void k_cast_f32_f64(const float* x, double* y, int32_t n) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        y[r] = (double)x[r];
}

int32_t launch_cast_f64_f32(const double* x, float* y, int32_t n, cudaStream_t s) {
    const int grid = max(1, min((n + 255) / 256, grid_cap(8)));
    k_cast_f64_f32<<<grid, 256, 0, s>>>(x, y, n);
    ++g_launches;
    return check_launch("k_cast_f64_f32");
}
int32_t launch_cast_f32_f64(const float* x, double* y, int32_t n, cudaStream_t s) {
    const int grid = max(1, min((n + 255) / 256, grid_cap(8)));
    k_cast_f32_f64<<<grid, 256, 0, s>>>(x, y, n);
    ++g_launches;
    return check_launch("k_cast_f32_f64");
}

__global__ void k_fill(double* x, double v, int32_t n) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        x[r] = v;
}
int32_t launch_fill(double* x, double v, int32_t n, cudaStream_t s) {
    const int grid = max(1, min((n + 255) / 256, grid_cap(8)));
    k_fill<<<grid, 256, 0, s>>>(x, v, n);
    ++g_launches;
    return check_launch("k_fill");
}

// out = a x + b y  (y may be null when b == 0)
template <typename T>
__global__ void k_axpby(T a, const T* x, T b, const T* y, T* out, int32_t n) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        out[r] = (y ? b * y[r] : T(0)) + a * x[r];
}
template <typename T>
int32_t launch_axpby(T a, const T* x, T b, const T* y, T* out, int32_t n, cudaStream_t s) {
    const int grid = max(1, min((n + 255) / 256, grid_cap(8)));
    k_axpby<T><<<grid, 256, 0, s>>>(a, x, b, y, out, n);
    ++g_launches;
    return check_launch("k_axpby");
}
template int32_t launch_axpby<double>(double, const double*, double, const double*,
                                      double*, int32_t, cudaStream_t);
template int32_t launch_axpby<float>(float, const float*, float, const float*, float*,
                                     int32_t, cudaStream_t);

}  // namespace ppg
