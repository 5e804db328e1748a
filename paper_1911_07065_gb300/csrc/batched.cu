// Batching form: many independent systems, each with its own GMRES
// polynomial, with one or four right-hand sides per system, solved together
// by flexible GMRES(m) in FP64 with p(A) v applied by Algorithm 3 in FP32
// (the precision form), the polynomials built by one batched GMRES(d) run.
//
// Layout.  The systems are packed into one block-diagonal CSR.  Each system
// starts on a 256-row tile (its rows are padded with empty rows), so every
// tile belongs to exactly one system and per-system reductions are sums
// over a contiguous range of tiles.  Vectors of the batch interleave the
// right-hand sides: element (row r, rhs k) sits at r * NR + k, so one pass
// over a matrix row serves all NR solves of its system (float4 / double2
// gathers).
//
// Polynomials.  Each system's Algorithm 3 chain (its own roots, real or
// paired, its own length) becomes a column of a step table; shorter chains
// are padded with no-op steps.  Pass k of the batch applies, in one launch,
// step k of every system: a CTA's rows all belong to one system, so the
// step it applies is uniform over the CTA.
//
// Krylov part.  CGS2 runs as in the single-system solver, with the dot
// products reduced per unit of up to 8 tiles and then per system in a fixed
// order (deterministic); one thread per solve applies the Givens rotations
// and decides on the device whether its solve stops in this cycle, so no
// step needs the host.  CTAs of a system whose solves have all stopped
// return at once, so converged systems cost next to nothing in later steps
// and cycles.
//
// Launch shape.  By default the whole solve, every restart cycle, runs in
// one persistent cooperative kernel (k_bpersist, its phases separated by
// bounded grid barriers); alternatively one restart cycle is captured once
// as a CUDA graph of the per-phase kernels and replayed for every cycle.
//
// Tiling.  The rows per CTA of the graph form's FP32 root-step kernel (64,
// 128 or 256) are chosen by timing the candidates on the batch at set-up;
// the persistent kernel runs its root steps on row groups of 64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ppg_common.cuh"

namespace ppg {
namespace {

constexpr int BT = 256;          // tile rows; every system starts on a tile
constexpr int OP_NOP = -2;
constexpr int OP_AXPY_B = -1;    // the elementwise step of a degree-one plan
constexpr int BCH = 8;           // columns per dot chunk
constexpr int BCHUNK = 2048;     // nonzeros staged per chunk
constexpr int BUNIT = 8;         // tiles per CTA of the batched CGS2 passes

struct BStep {
    int op, flags;
    double c1, c2, c3;
    int x, a0, a1, a2, o0, o1;
};

template <typename T>
struct BufSet {
    T* p[6];
};

// ---------------------------------------------------------------------------
// vector loads of the NR interleaved right-hand sides of one row
// ---------------------------------------------------------------------------

template <typename T, int NR>
__device__ __forceinline__ void ld_rhs(const T* p, T (&out)[NR]) {
    if constexpr (NR == 4 && sizeof(T) == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p));
        out[0] = q.x; out[1] = q.y; out[2] = q.z; out[3] = q.w;
    } else if constexpr (NR == 4 && sizeof(T) == 8) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
        out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
    } else {
#pragma unroll
        for (int i = 0; i < NR; ++i) out[i] = __ldg(p + i);
    }
}

// does any right-hand side of system s still take steps in this cycle?
template <int NR>
__device__ __forceinline__ bool sys_live(const int32_t* active, int s) {
    int any = 0;
#pragma unroll
    for (int k = 0; k < NR; ++k) any |= active[s * NR + k];
    return any != 0;
}

// Synchronise the `rows` threads of one row group: the whole CTA when the
// group is the CTA, else a named barrier of the group (ids 1..4; barrier 0
// is __syncthreads).
__device__ __forceinline__ void group_sync(int group, int rows) {
    if (rows == (int)blockDim.x) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(group + 1), "r"(rows) : "memory");
    }
}

// One tile of one pass of the batch: step steps[s] of system s (the owner of
// the tile) applied to the NR right-hand sides of `rows` consecutive rows,
// one thread (gt) per row.  Ops as in the single-system kernel; OP_NOP
// leaves everything untouched.  OP_RESID writes the tile's partial sums of
// squares, part[vt * NR + k] (only with rows == blockDim.x).  The staging
// buffers sval / scol hold `chunk` nonzeros, srp rows + 1 row pointers.
template <typename T, int NR>
__device__ __forceinline__ void bstep_tile(
    int64_t vt, int rows, int gt, int group, T* sval, int32_t* scol, int32_t* srp, int chunk,
    double (*sred)[NR], const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
    const T* __restrict__ vals, const BStep* __restrict__ steps,
    const int32_t* __restrict__ sys_of_tile, const BufSet<T>& b, double* part,
    const int32_t* __restrict__ active) {
    const int tid = gt;
    const int64_t row0 = vt * rows;
    const int s = sys_of_tile[row0 / BT];
    const BStep st = steps[s];
    if (st.op == OP_NOP) return;   // uniform over the group
    if (active && !sys_live<NR>(active, s)) return;   // every solve of s has stopped
    for (int i = tid; i <= rows; i += rows) srp[i] = __ldg(rowptr + row0 + i);
    group_sync(group, rows);
    const int32_t k0 = srp[0], k1 = srp[rows];
    const int32_t lo_r = srp[tid], hi_r = srp[tid + 1];
    const int64_t r = row0 + tid;
    const T* x = b.p[st.x];
    T e0[NR], e1[NR], e2[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) e0[i] = e1[i] = e2[i] = T(0);
    if (st.a0 >= 0) ld_rhs<T, NR>(b.p[st.a0] + r * NR, e0);
    if (st.a1 >= 0 && !(st.flags & F_PZERO))
#pragma unroll
        for (int i = 0; i < NR; ++i) e1[i] = b.p[st.a1][r * NR + i];
    if (st.a2 >= 0 && (st.flags & F_FINAL)) ld_rhs<T, NR>(b.p[st.a2] + r * NR, e2);

    T acc[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) acc[i] = T(0);
    for (int32_t c0 = k0; c0 < k1; c0 += chunk) {
        const int32_t c1 = min(k1, c0 + chunk);
        // asynchronous, coalesced staging of the tile's values and columns
        for (int32_t k = c0 + tid; k < c1; k += rows) {
            const unsigned sv_ = (unsigned)__cvta_generic_to_shared(sval + (k - c0));
            const unsigned sc_ = (unsigned)__cvta_generic_to_shared(scol + (k - c0));
            asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sv_), "l"(vals + k),
                         "n"(sizeof(T)) : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sc_), "l"(colind + k)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        group_sync(group, rows);
        const int32_t lo = max(lo_r, c0) - c0, hi = min(hi_r, c1) - c0;
        int32_t k = lo;
        // one FMA per nonzero and right-hand side, the gathers of two
        // nonzeros (2 NR values) in flight before their multiply-adds
        for (; k + 2 <= hi; k += 2) {
            T x0[NR], x1[NR];
            ld_rhs<T, NR>(x + (int64_t)scol[k] * NR, x0);
            ld_rhs<T, NR>(x + (int64_t)scol[k + 1] * NR, x1);
            const T v0 = sval[k], v1 = sval[k + 1];
#pragma unroll
            for (int i = 0; i < NR; ++i) acc[i] = fma(v1, x1[i], fma(v0, x0[i], acc[i]));
        }
        if (k < hi) {
            T x0[NR];
            ld_rhs<T, NR>(x + (int64_t)scol[k] * NR, x0);
            const T v0 = sval[k];
#pragma unroll
            for (int i = 0; i < NR; ++i) acc[i] = fma(v0, x0[i], acc[i]);
        }
        group_sync(group, rows);
    }
    const T c1 = (T)st.c1, c2 = (T)st.c2, c3 = (T)st.c3;
    T* o0 = st.o0 >= 0 ? b.p[st.o0] + r * NR : nullptr;
    if (st.op == OP_AXPY_B) {   // degree-one polynomial: P = c1 v (+ P)
        T xr[NR];
        ld_rhs<T, NR>(x + r * NR, xr);
#pragma unroll
        for (int i = 0; i < NR; ++i)
            o0[i] = (st.flags & F_PZERO) ? c1 * xr[i] : fma(c1, xr[i], e1[i]);
        return;
    }
    T* o1 = st.o1 >= 0 ? b.p[st.o1] + r * NR : nullptr;
    double sq[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        sq[i] = 0.0;
        const T s_ = acc[i];
        if (st.op == OP_SPMV) {
            o0[i] = s_;
        } else if (st.op == OP_RESID) {
            const T v = e0[i] - s_;
            o0[i] = v;
            sq[i] = (double)v * (double)v;
        } else if (st.op == OP_P_REAL) {
            const T pnew = (st.flags & F_PZERO) ? c1 * e0[i] : fma(c1, e0[i], e1[i]);
            const T prodn = fma(-c1, s_, e0[i]);
            if (st.flags & F_FINAL) {
                o0[i] = fma(c3, prodn, pnew);
            } else {
                o0[i] = pnew;
                o1[i] = prodn;
            }
        } else if (st.op == OP_P_PAIR1) {
            const T tmp = fma(c1, e0[i], -s_);
            o0[i] = (st.flags & F_PZERO) ? c2 * tmp : fma(c2, tmp, e1[i]);
            if (!(st.flags & F_NO_O1)) o1[i] = tmp;
        } else if (st.op == OP_P_PAIR2) {
            const T prodn = fma(-c2, s_, e0[i]);
            o0[i] = (st.flags & F_FINAL) ? fma(c3, prodn, e1[i]) : prodn;
        }
    }
    if (st.op == OP_RESID) {
        const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            double v = sq[i];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) sred[warp][i] = v;
        }
        group_sync(group, rows);
        if (tid < NR) {
            double t = 0.0;
            for (int w = 0; w < (rows >> 5); ++w) t += sred[w][tid];
            part[(size_t)vt * NR + tid] = t;
        }
    }
}

// One pass of the batch over all tiles: one CTA per tile of blockDim.x rows.
// Register bound: 32 per thread (8 CTAs of 256 threads per SM) for the FP32
// steps and the one-rhs FP64 step, measured 3 % faster on the batching
// workload than the 40 registers the FP32 step takes unbounded; the FP64
// four-rhs step would spill at 32.
template <typename T, int NR>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 || NR == 1) ? 8 : 4)
k_bstep(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
        const T* __restrict__ vals, const BStep* __restrict__ steps,
        const int32_t* __restrict__ sys_of_tile, BufSet<T> b, double* part,
        const int32_t* __restrict__ active) {
    __shared__ T sval[BCHUNK];
    __shared__ int32_t scol[BCHUNK];
    __shared__ int32_t srp[BT + 1];
    __shared__ double sred[8][NR];
    bstep_tile<T, NR>(blockIdx.x, blockDim.x, threadIdx.x, 0, sval, scol, srp, BCHUNK, sred,
                      rowptr, colind, vals, steps, sys_of_tile, b, part, active);
}

template <int NR, int NQ>
__device__ __forceinline__ void bdot_unit(const double* const* col, const double* __restrict__ w,
                                          int t0, int t1, int tid, int k, double* acc) {
    constexpr int RP = 256 / NR;   // rows per pass
#pragma unroll 2
    for (int t = t0; t < t1; ++t) {
        const int64_t base = (int64_t)t * BT;
#pragma unroll
        for (int p = 0; p < NR; ++p) {
            const int64_t idx = (base + p * RP + tid / NR) * NR + k;
            const double wv = w[idx];
#pragma unroll
            for (int q = 0; q < NQ; ++q) acc[q] = fma(__ldcs(col[q] + idx), wv, acc[q]);
        }
    }
}

// Partial dot products per unit (up to BUNIT consecutive tiles of one
// system): part[unit * pstr + c * NR + k] = sum over the unit's rows of
// col_c[r, k] * w[r, k], where col_c is basis column c (c < ncol) or w
// itself (c == ncol, with_self), for the columns of chunk cy (BCH columns
// from cy * BCH).  Thread t takes rhs k = t % NR of rows t / NR,
// t / NR + 256 / NR, ... of every tile of the unit.  256 threads.
template <int NR>
__device__ __forceinline__ void bdot_block(int unit, int cy, double (*sred)[BCH][NR],
                                           const double* __restrict__ V, int64_t ldV, int ncol,
                                           const double* __restrict__ w, int with_self,
                                           double* part, int64_t pstr,
                                           const int32_t* __restrict__ unit_tile0,
                                           const int32_t* __restrict__ sys_of_unit,
                                           const int32_t* __restrict__ active) {
    // stopped systems: their partial sums are never read
    if (active && !sys_live<NR>(active, sys_of_unit[unit])) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int k = tid % NR;
    const int t0 = unit_tile0[unit], t1 = unit_tile0[unit + 1];
    const int c0 = cy * BCH;
    const int nvals = ncol + (with_self ? 1 : 0);
    const int nq = min(BCH, nvals - c0);
    const double* col[BCH];
#pragma unroll
    for (int q = 0; q < BCH; ++q) {
        const int c = c0 + q;
        col[q] = (c < ncol) ? V + c * ldV : w;
    }
    double acc[BCH];
#pragma unroll
    for (int q = 0; q < BCH; ++q) acc[q] = 0.0;
    switch (nq) {   // compile-time widths: no FP64 FMA for a missing column
        case 8: bdot_unit<NR, 8>(col, w, t0, t1, tid, k, acc); break;
        case 7: bdot_unit<NR, 7>(col, w, t0, t1, tid, k, acc); break;
        case 6: bdot_unit<NR, 6>(col, w, t0, t1, tid, k, acc); break;
        case 5: bdot_unit<NR, 5>(col, w, t0, t1, tid, k, acc); break;
        case 4: bdot_unit<NR, 4>(col, w, t0, t1, tid, k, acc); break;
        case 3: bdot_unit<NR, 3>(col, w, t0, t1, tid, k, acc); break;
        case 2: bdot_unit<NR, 2>(col, w, t0, t1, tid, k, acc); break;
        default: bdot_unit<NR, 1>(col, w, t0, t1, tid, k, acc); break;
    }
    // sum over the lanes that share k
#pragma unroll
    for (int q = 0; q < BCH; ++q)
        for (int off = NR; off < 32; off <<= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
    if (lane < NR)
#pragma unroll
        for (int q = 0; q < BCH; ++q) sred[warp][q][lane] = acc[q];
    __syncthreads();
    if (tid < BCH * NR) {
        const int q = tid / NR, kk = tid % NR;
        if (c0 + q < nvals) {
            double t = 0.0;
#pragma unroll
            for (int ww = 0; ww < 8; ++ww) t += sred[ww][q][kk];
            part[(size_t)unit * pstr + (c0 + q) * NR + kk] = t;
        }
    }
}

template <int NR>
__global__ void __launch_bounds__(256)
k_bdot(const double* __restrict__ V, int64_t ldV, int ncol, const double* __restrict__ w,
       int with_self, double* part, int64_t pstr, const int32_t* __restrict__ unit_tile0,
       const int32_t* __restrict__ sys_of_unit, const int32_t* __restrict__ active) {
    __shared__ double sred[8][BCH][NR];
    bdot_block<NR>(blockIdx.x, blockIdx.y, sred, V, ldV, ncol, w, with_self, part, pstr,
                   unit_tile0, sys_of_unit, active);
}

// out[c * nsolve + s * NR + k] = sum over units u of system s (in order) of
// part[u * pstr + c * NR + k], for c < nvals.  One warp per (s, c): the
// block (s, cy) takes c = cy * 8 + warp.
__device__ __forceinline__ void bsegsum_block(int s, int cy, const double* part, int64_t pstr,
                                              int nvals, int NR, const int32_t* unit0,
                                              int nsys, double* out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = cy * 8 + warp;
    if (s >= nsys || c >= nvals) return;
    const int u0 = unit0[s], u1 = unit0[s + 1];
    const int nsolve = nsys * NR;
    for (int k = 0; k < NR; ++k) {
        double t = 0.0;
        for (int u = u0 + lane; u < u1; u += 32) t += part[(size_t)u * pstr + c * NR + k];
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) out[(size_t)c * nsolve + s * NR + k] = t;
    }
}

__global__ void k_bsegsum(const double* part, int64_t pstr, int nvals, int NR,
                          const int32_t* unit0, int nsys, double* out) {
    bsegsum_block(blockIdx.x, blockIdx.y, part, pstr, nvals, NR, unit0, nsys, out);
}

// w[r, k] -= sum_c V_c[r, k] h[c, solve(r, k)] over the rows of one unit
// per block; with_norm: per-unit partial sums of the new w[r, k]^2 in
// part[unit * NR + k].  256 threads.
template <int NR>
__device__ __forceinline__ void bsub_block(int unit, double (*sh)[NR], double (*sred)[NR],
                                           const double* __restrict__ V, int64_t ldV, int ncol,
                                           double* w, const double* __restrict__ h, int nsolve,
                                           const int32_t* __restrict__ unit_tile0,
                                           const int32_t* __restrict__ sys_of_unit,
                                           int with_norm, double* part,
                                           const int32_t* __restrict__ active) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int k = tid % NR;
    constexpr int RP = 256 / NR;
    const int s = sys_of_unit[unit];
    if (active && !sys_live<NR>(active, s)) return;
    const int t0 = unit_tile0[unit], t1 = unit_tile0[unit + 1];
    for (int e = tid; e < ncol * NR; e += 256)
        sh[e / NR][e % NR] = h[(size_t)(e / NR) * nsolve + s * NR + e % NR];
    __syncthreads();
    double nacc = 0.0;
    for (int t = t0; t < t1; ++t) {
        const int64_t base = (int64_t)t * BT;
        // the NR rows of this thread in the tile share each coefficient load:
        // column pairs outermost (even columns into s0, odd into s1, as a
        // per-row loop would sum them), the rows innermost
        const int64_t idx0 = (base + tid / NR) * NR + k;
        double s0[NR], s1[NR];
#pragma unroll
        for (int p = 0; p < NR; ++p) s0[p] = s1[p] = 0.0;
        int c = 0;
        for (; c + 1 < ncol; c += 2) {
            const double h0 = sh[c][k], h1 = sh[c + 1][k];
            const double* v0 = V + c * ldV + idx0;
            const double* v1 = V + (c + 1) * ldV + idx0;
#pragma unroll
            for (int p = 0; p < NR; ++p) {
                s0[p] = fma(__ldcs(v0 + p * RP * NR), h0, s0[p]);
                s1[p] = fma(__ldcs(v1 + p * RP * NR), h1, s1[p]);
            }
        }
        if (c < ncol) {
            const double h0 = sh[c][k];
            const double* v0 = V + c * ldV + idx0;
#pragma unroll
            for (int p = 0; p < NR; ++p) s0[p] = fma(__ldcs(v0 + p * RP * NR), h0, s0[p]);
        }
#pragma unroll
        for (int p = 0; p < NR; ++p) {
            const int64_t idx = idx0 + (int64_t)p * RP * NR;
            const double wn = w[idx] - (s0[p] + s1[p]);
            w[idx] = wn;
            nacc = fma(wn, wn, nacc);
        }
    }
    if (!with_norm) return;
    for (int off = NR; off < 32; off <<= 1) nacc += __shfl_xor_sync(0xffffffffu, nacc, off);
    if (lane < NR) sred[warp][lane] = nacc;
    __syncthreads();
    if (tid < NR) {
        double t = 0.0;
        for (int ww = 0; ww < 8; ++ww) t += sred[ww][tid];
        part[(size_t)unit * NR + tid] = t;
    }
}

template <int NR>
__global__ void __launch_bounds__(256)
k_bsub(const double* __restrict__ V, int64_t ldV, int ncol, double* w,
       const double* __restrict__ h, int nsolve, const int32_t* __restrict__ unit_tile0,
       const int32_t* __restrict__ sys_of_unit, int with_norm, double* part,
       const int32_t* __restrict__ active) {
    __shared__ double sh[ORTHO_MAXC][NR];
    __shared__ double sred[8][NR];
    bsub_block<NR>(blockIdx.x, sh, sred, V, ldV, ncol, w, h, nsolve, unit_tile0, sys_of_unit,
                   with_norm, part, active);
}

struct BState {      // device, per solve (nsolve = nsys * NR)
    double* R;       // [nsolve][ldh * m]
    double* Hraw;    // [nsolve][ldh * m] (construction)
    double* cs;      // [nsolve][m]
    double* sn;
    double* g;       // [nsolve][m + 1]
    double* y;       // [nsolve][m]
    double* inv;     // [nsolve] scale of the next basis vector
    double* bnorm;   // [nsolve]
    double* relres;  // [nsolve] true relative residual after the last cycle
    int32_t* active; // [nsolve] the solve takes Arnoldi steps in this cycle
    int32_t* ksteps; // [nsolve] steps taken in this cycle
    int32_t* iters;  // [nsolve] total steps
    int32_t* brk;    // [nsolve] construction: first breakdown step, -1 none
};

// One Arnoldi step for every solve: Hessenberg column from h1 + h2 and
// ||w||^2; construction mode stores Hbar and detects breakdown
// (h <= 1e-13 ||A v_j||); solve mode applies the rotations, updates g and
// stops the solve (for this cycle) when the shortcut residual reaches tol,
// on breakdown, or at the cycle's last step.
__device__ __forceinline__ void bgivens_one(int sv, const BState& st, int nsolve, int ldh, int m,
                                            int j, const double* h1, const double* h2,
                                            const double* nrm, int build, double tol) {
    if (!st.active[sv]) {
        st.inv[sv] = 0.0;
        return;
    }
    double col[ORTHO_MAXC + 1];
    for (int i = 0; i <= j; ++i) col[i] = h1[(size_t)i * nsolve + sv] + h2[(size_t)i * nsolve + sv];
    const double hn = sqrt(fmax(nrm[sv], 0.0));
    col[j + 1] = hn;
    if (build) {
        double* H = st.Hraw + (size_t)sv * ldh * m;
        for (int i = 0; i <= j + 1; ++i) H[(size_t)j * ldh + i] = col[i];
        const double w0 = sqrt(fmax(h1[(size_t)(j + 1) * nsolve + sv], 0.0));
        if (!(hn > 1e-13 * w0)) {
            H[(size_t)j * ldh + j + 1] = 0.0;
            st.brk[sv] = j;
            st.active[sv] = 0;
            st.inv[sv] = 0.0;
            st.ksteps[sv] = j + 1;
        } else {
            st.inv[sv] = 1.0 / hn;
            st.ksteps[sv] = j + 1;
        }
        return;
    }
    double* cs = st.cs + (size_t)sv * m;
    double* sn = st.sn + (size_t)sv * m;
    double* g = st.g + (size_t)sv * (m + 1);
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
    }
    const double a = col[j], bb = col[j + 1];
    const double r = hypot(a, bb);
    double c = 1.0, s = 0.0;
    if (r != 0.0) { c = a / r; s = bb / r; }
    cs[j] = c;
    sn[j] = s;
    col[j] = r;
    double* R = st.R + (size_t)sv * ldh * m;
    for (int i = 0; i <= j; ++i) R[(size_t)j * ldh + i] = col[i];
    const double gj = g[j];
    g[j + 1] = -s * gj;
    g[j] = c * gj;
    const double est = fabs(g[j + 1]) / st.bnorm[sv];
    if (est <= tol || !(hn > 0.0) || j + 1 == m || !isfinite(est)) {
        st.active[sv] = 0;
        st.ksteps[sv] = j + 1;
        st.inv[sv] = 0.0;
    } else {
        st.inv[sv] = 1.0 / hn;
    }
}

__global__ void k_bgivens(BState st, int nsolve, int ldh, int m, int j, const double* h1,
                          const double* h2, const double* nrm, int build, double tol) {
    const int sv = blockIdx.x * blockDim.x + threadIdx.x;
    if (sv < nsolve) bgivens_one(sv, st, nsolve, ldh, m, j, h1, h2, nrm, build, tol);
}

// w[r, k] *= scale[solve(r, k)] for elements e = e0, e0 + stride, ...; with
// w32, also its FP32 copy, which the next Arnoldi step's Algorithm 3 chain
// reads (the scaling of a basis column and that cast in one pass)
template <int NR>
__device__ __forceinline__ void bscale_range(double* w, const double* scale,
                                             const int32_t* sys_of_tile, int64_t total,
                                             int64_t e0, int64_t stride, float* w32) {
    for (int64_t e = e0; e < total; e += stride) {
        const int64_t row = e / NR;
        const int sv = sys_of_tile[row / BT] * NR + (int)(e % NR);
        const double t = w[e] * scale[sv];
        w[e] = t;
        if (w32) w32[e] = (float)t;
    }
}

template <int NR>
__global__ void k_bscale(double* w, const double* scale, const int32_t* sys_of_tile,
                         int64_t total, float* w32) {
    bscale_range<NR>(w, scale, sys_of_tile, total, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                     (int64_t)gridDim.x * blockDim.x, w32);
}

// one warp per solve: row i from the bottom up, the lanes sharing the sum
// over the solved entries c > i, lane 0 dividing
__device__ __forceinline__ void bbacksolve_warp(int sv, int lane, const BState& st, int ldh,
                                                int m) {
    const int k = st.ksteps[sv];
    const double* R = st.R + (size_t)sv * ldh * m;
    const double* g = st.g + (size_t)sv * (m + 1);
    double* y = st.y + (size_t)sv * m;
    for (int i = k - 1; i >= 0; --i) {
        double part = 0.0;
        for (int c = i + 1 + lane; c < k; c += 32) part = fma(R[(size_t)c * ldh + i], y[c], part);
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        if (lane == 0) y[i] = (g[i] - part) / R[(size_t)i * ldh + i];
        __syncwarp();
    }
}

__global__ void k_bbacksolve(BState st, int nsolve, int ldh, int m) {
    const int sv = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (sv < nsolve) bbacksolve_warp(sv, threadIdx.x & 31, st, ldh, m);   // uniform per warp
}

// x[r, k] += sum_{c < ksteps} Z_c[r, k] y[solve][c]
template <int NR>
__device__ __forceinline__ void bzy_range(const float* __restrict__ Z, int64_t ldZ, double* x,
                                          const BState& st,
                                          const int32_t* __restrict__ sys_of_tile, int m,
                                          int64_t total, int64_t e0, int64_t stride) {
    for (int64_t e = e0; e < total; e += stride) {
        const int64_t row = e / NR;
        const int sv = sys_of_tile[row / BT] * NR + (int)(e % NR);
        const int k = st.ksteps[sv];
        const double* y = st.y + (size_t)sv * m;
        double s = x[e];
        for (int c = 0; c < k; ++c) s = fma((double)__ldcs(Z + c * ldZ + e), y[c], s);
        x[e] = s;
    }
}

template <int NR>
__global__ void k_bzy(const float* __restrict__ Z, int64_t ldZ, double* x, BState st,
                      const int32_t* __restrict__ sys_of_tile, int m, int64_t total) {
    bzy_range<NR>(Z, ldZ, x, st, sys_of_tile, m, total,
                  (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                  (int64_t)gridDim.x * blockDim.x);
}

// After a true residual: beta per solve, relres, the next cycle's g[0],
// the scale of V_0, and which solves take steps in the next cycle.
__device__ __forceinline__ void bcycle_one(int sv, const BState& st, int m, const double* nrm2,
                                           double tol, int first) {
    const double beta = sqrt(fmax(nrm2[sv], 0.0));
    if (first) st.bnorm[sv] = beta;
    if (!first) st.iters[sv] += st.ksteps[sv];
    const double bn = st.bnorm[sv];
    const double rel = bn > 0.0 ? beta / bn : 0.0;
    st.relres[sv] = rel;
    st.g[(size_t)sv * (m + 1)] = beta;
    st.ksteps[sv] = 0;
    const bool go = bn > 0.0 && rel > tol && isfinite(rel);
    st.active[sv] = go ? 1 : 0;
    st.inv[sv] = (go && beta > 0.0) ? 1.0 / beta : 0.0;
}

__global__ void k_bcycle(BState st, int nsolve, int m, const double* nrm2, double tol,
                         int first) {
    const int sv = blockIdx.x * blockDim.x + threadIdx.x;
    if (sv < nsolve) bcycle_one(sv, st, m, nrm2, tol, first);
}

// ---------------------------------------------------------------------------
// packing
// ---------------------------------------------------------------------------

__global__ void k_pack_csr(const int32_t* rowptr, const int32_t* colind, const double* vals,
                           int32_t n, int32_t np, int64_t row_off, int64_t nnz_off,
                           int32_t* prow, int32_t* pcol, double* p64, float* p32) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = t; i < np; i += stride)
        prow[row_off + i] = (int32_t)(nnz_off + rowptr[i < n ? i : n]);
    const int32_t nnz = rowptr[n];
    for (int64_t k = t; k < nnz; k += stride) {
        pcol[nnz_off + k] = (int32_t)(row_off + colind[k]);
        p64[nnz_off + k] = vals[k];
        p32[nnz_off + k] = (float)vals[k];
    }
}

// packed[(row_off + i) * NR + k] = src[k * n + i] (src column-major n x NR)
__global__ void k_pack_vec(const double* src, int32_t n, int32_t np, int NR, int64_t row_off,
                           double* dst, int nr_src) {
    const int64_t total = (int64_t)np * NR;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / NR;
        const int k = (int)(e % NR);
        dst[(row_off + i) * NR + k] = (i < n && k < nr_src) ? src[(int64_t)k * n + i] : 0.0;
    }
}

__global__ void k_unpack_vec(const double* src, int32_t n, int NR, int64_t row_off, double* dst,
                             int nr_dst) {
    const int64_t total = (int64_t)n * nr_dst;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n;
        const int k = (int)(e / n);
        dst[e] = src[(row_off + i) * NR + k];
    }
}

__global__ void k_cast32(const float* x, double* y, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        y[e] = (double)x[e];
}

// ---------------------------------------------------------------------------
// The whole solve in one persistent launch
// ---------------------------------------------------------------------------
//
// k_bpersist runs every restart cycle of every solve of the batch: the same
// phases as the per-cycle graph (FP32 cast, the Algorithm 3 root steps, the
// FP64 operator product, the CGS2 unit passes, the Givens updates, the
// scaling; at a cycle's end the back substitution, x += Z y, the true
// residual and the restart), each phase a loop of the CTA over virtual
// blocks, the phases separated by grid-wide barriers.  It is launched
// cooperatively, so every CTA is resident and the barriers cannot wait for
// a CTA that has not started.  Each barrier wait is bounded by a time limit;
// a CTA whose wait runs out raises the shared error flag and returns, and
// every other CTA returns at its next barrier (PPG_ERR_TIMEOUT on the host).
// The FP32 root steps run on row groups of `rows` threads (64, 128 or 256,
// the autotuned row tiling), several groups per CTA, each on its own tile
// with its own staging slice and named barrier.

struct GridBar {
    unsigned count;   // CTAs arrived at the current barrier
    unsigned gen;     // barriers completed
    unsigned err;     // a wait ran out
    unsigned pad;
};

struct PArgs {
    const int32_t* rowptr;
    const int32_t* colind;
    const double* v64;
    const float* v32;
    const int32_t* sys_of_tile;
    const int32_t* unit_tile0;
    const int32_t* unit0;
    const int32_t* sys_of_unit;
    const int32_t* cta0;
    int nsys, m, ldh, K, max_cycles, rows;
    int64_t N, nunits, ntiles;
    double tol;
    double* V;
    float* Z;
    float *fa, *fb, *fc, *x32;
    double* zd;
    double* X;
    double* Bp;
    double* part;
    int64_t pstr;
    double *h1, *h2, *nrm;
    const BStep* steps_p;
    const BStep* steps_spmv;
    const BStep* steps_resid;
    BState st;
    GridBar* bar;
    unsigned long long timeout_ns;
    int32_t* cycles_out;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch.  Thread 0 of each CTA arrives
// on the counter; the last to arrive resets it and advances the
// generation, the others wait for the generation to move, at most
// timeout_ns (and a bounded number of polls).  Returns false, uniformly
// over the CTA, when this or any other CTA's wait ran out.
__device__ bool grid_sync(GridBar* gb, unsigned long long timeout_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = &gb->gen;
        volatile unsigned* verr = &gb->err;
        int ok = 1;
        const unsigned g0 = *vgen;
        __threadfence();
        if (atomicAdd(&gb->count, 1u) == gridDim.x - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            for (unsigned it = 0; *vgen == g0; ++it) {
                if (*verr != 0u) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > timeout_ns || it > (1u << 28)) {
                    atomicExch(&gb->err, 1u);
                    ok = 0;
                    break;
                }
                if (it > 64) __nanosleep(32);   // spin briefly before backing off
            }
        }
        if (*verr != 0u) ok = 0;
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// does any solve still take steps?  (all CTAs read the same array after a
// barrier, so the answer is uniform over the grid)
__device__ __forceinline__ bool any_active(const int32_t* active, int nsolve) {
    __shared__ int s_any;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    int mine = 0;
    for (int i = threadIdx.x; i < nsolve; i += blockDim.x) mine |= active[i];
    if (mine) s_any = 1;
    __syncthreads();
    const bool r = s_any != 0;
    __syncthreads();
    return r;
}

#define PSYNC()                                             \
    do {                                                    \
        if (!grid_sync(a.bar, a.timeout_ns)) return;        \
    } while (0)

template <int NR>
__global__ void __launch_bounds__(256, 4) k_bpersist(const PArgs a) {
    // staging shared by the root-step phases (FP32: values then columns,
    // sliced per row group; FP64: the whole CTA)
    __shared__ __align__(16) unsigned char sraw[BCHUNK * (8 + 4)];
    __shared__ int32_t srp[BT + 8];
    __shared__ double sred[8][NR];
    __shared__ double bd_sred[8][BCH][NR];
    __shared__ double bs_sh[ORTHO_MAXC][NR];
    const int tid = threadIdx.x, lane = tid & 31;
    const int nsolve = a.nsys * NR;
    const int64_t total = a.N * NR;
    const int64_t ldV = total;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
    const int rows = a.rows;
    const int groups = 256 / rows;
    const int group = tid / rows, gt = tid % rows;
    const int fchunk = BCHUNK * rows / 256;
    float* fsval = reinterpret_cast<float*>(sraw) + group * fchunk;
    int32_t* fscol = reinterpret_cast<int32_t*>(sraw + BCHUNK * 4) + group * fchunk;
    int32_t* fsrp = srp + group * (rows + 1);
    double* dsval = reinterpret_cast<double*>(sraw);
    int32_t* dscol = reinterpret_cast<int32_t*>(sraw + BCHUNK * 8);
    const int64_t nvt_f = a.N / rows;   // tiles of `rows` rows in the batch
    int cycles = 0;
    for (int cyc = 0; cyc < a.max_cycles; ++cyc) {
        if (!any_active(a.st.active, nsolve)) break;
        ++cycles;
        for (int j = 0; j < a.m; ++j) {
            double* w = a.V + (size_t)(j + 1) * ldV;
            float* zj = a.Z + (size_t)j * ldV;
            // z_j = p(A) v_j: Algorithm 3 in FP32, one pass per step (its FP32
            // copy x32 of v_j was written with the scaling of v_j)
            BufSet<float> fs{};
            fs.p[B_IN] = a.x32;
            fs.p[B_P] = zj;
            fs.p[B_A] = a.fa;
            fs.p[B_B] = a.fb;
            fs.p[B_C] = a.fc;
            for (int k = 0; k < a.K; ++k) {
                const BStep* steps = a.steps_p + (size_t)k * a.nsys;
                // each row group strides over the tiles on its own: the groups use
                // disjoint shared-memory slices and their own barriers
                for (int64_t vt = (int64_t)blockIdx.x * groups + group; vt < nvt_f;
                     vt += (int64_t)gridDim.x * groups)
                    bstep_tile<float, NR>(vt, rows, gt, group, fsval, fscol, fsrp, fchunk, sred,
                                          a.rowptr, a.colind, a.v32, steps, a.sys_of_tile, fs,
                                          nullptr, a.st.active);
                PSYNC();
            }
            for (int64_t e = gtid; e < total; e += gstride) a.zd[e] = (double)zj[e];
            PSYNC();
            // w = A z_j in FP64
            BufSet<double> ds{};
            ds.p[B_IN] = a.zd;
            ds.p[B_OUT] = w;
            for (int64_t vb = blockIdx.x; vb < a.ntiles; vb += gridDim.x) {
                bstep_tile<double, NR>(vb, 256, tid, 0, dsval, dscol, srp, BCHUNK, sred, a.rowptr,
                                       a.colind, a.v64, a.steps_spmv, a.sys_of_tile, ds, nullptr,
                                       a.st.active);
                __syncthreads();
            }
            PSYNC();
            // CGS2 over the j + 1 basis columns, per unit, reduced per system
            const int ncol = j + 1;
            const int nch = (ncol + BCH - 1) / BCH;
            for (int pass = 0; pass < 2; ++pass) {
                double* h = pass == 0 ? a.h1 : a.h2;
                for (int64_t vb = blockIdx.x; vb < a.nunits * nch; vb += gridDim.x) {
                    bdot_block<NR>((int)(vb % a.nunits), (int)(vb / a.nunits), bd_sred, a.V, ldV,
                                   ncol, w, 0, a.part, a.pstr, a.unit_tile0, a.sys_of_unit,
                                   a.st.active);
                    __syncthreads();
                }
                PSYNC();
                const int nseg = a.nsys * ((ncol + 7) / 8);
                for (int vb = blockIdx.x; vb < nseg; vb += gridDim.x)
                    bsegsum_block(vb % a.nsys, vb / a.nsys, a.part, a.pstr, ncol, NR, a.unit0,
                                  a.nsys, h);
                PSYNC();
                for (int64_t vb = blockIdx.x; vb < a.nunits; vb += gridDim.x) {
                    bsub_block<NR>((int)vb, bs_sh, sred, a.V, ldV, ncol, w, h, nsolve,
                                   a.unit_tile0, a.sys_of_unit, pass == 1, a.part, a.st.active);
                    __syncthreads();
                }
                PSYNC();
            }
            for (int vb = blockIdx.x; vb < a.nsys; vb += gridDim.x)
                bsegsum_block(vb, 0, a.part, NR, 1, NR, a.unit0, a.nsys, a.nrm);
            PSYNC();
            for (int64_t sv = gtid; sv < nsolve; sv += gstride)
                bgivens_one((int)sv, a.st, nsolve, a.ldh, a.m, j, a.h1, a.h2, a.nrm, 0, a.tol);
            PSYNC();
            bscale_range<NR>(w, a.st.inv, a.sys_of_tile, total, gtid, gstride, a.x32);
            PSYNC();
            if (!any_active(a.st.active, nsolve)) break;
        }
        // end of the cycle: y = R^-1 g, x += Z y, r = b - A x, restart
        for (int64_t sv = gtid >> 5; sv < nsolve; sv += gstride >> 5)
            bbacksolve_warp((int)sv, lane, a.st, a.ldh, a.m);
        PSYNC();
        bzy_range<NR>(a.Z, ldV, a.X, a.st, a.sys_of_tile, a.m, total, gtid, gstride);
        PSYNC();
        BufSet<double> rs{};
        rs.p[B_IN] = a.X;
        rs.p[B_P] = a.Bp;
        rs.p[B_OUT] = a.V;
        for (int64_t vb = blockIdx.x; vb < a.ntiles; vb += gridDim.x) {
            bstep_tile<double, NR>(vb, 256, tid, 0, dsval, dscol, srp, BCHUNK, sred, a.rowptr,
                                   a.colind, a.v64, a.steps_resid, a.sys_of_tile, rs, a.part,
                                   nullptr);
            __syncthreads();
        }
        PSYNC();
        for (int vb = blockIdx.x; vb < a.nsys; vb += gridDim.x)
            bsegsum_block(vb, 0, a.part, NR, 1, NR, a.cta0, a.nsys, a.nrm);
        PSYNC();
        for (int64_t sv = gtid; sv < nsolve; sv += gstride)
            bcycle_one((int)sv, a.st, a.m, a.nrm, a.tol, 0);
        PSYNC();
        bscale_range<NR>(a.V, a.st.inv, a.sys_of_tile, total, gtid, gstride, a.x32);
        PSYNC();
    }
    if (blockIdx.x == 0 && tid == 0) *a.cycles_out = cycles;
}

#undef PSYNC

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

int elem_grid(int64_t total) {
    const int64_t g = (total + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, grid_cap(8)));
}

#define BCHECK(where)                                 \
    do {                                              \
        ++g_launches;                                 \
        int32_t rc__ = check_launch(where);           \
        if (rc__ < 0) return rc__;                    \
    } while (0)

struct Batch {
    int nsys = 0, NR = 1, m = 0, ldh = 0, d = 0;
    int64_t N = 0, nnz = 0, ntiles = 0;
    std::vector<int64_t> off;      // row offset per system
    std::vector<int32_t> n;        // rows per system
    std::vector<int32_t> tile0_h;  // first tile per system, nsys + 1
    // units of the CGS2 passes: up to BUNIT consecutive tiles of one system
    int64_t nunits = 0;
    std::vector<int32_t> unit_tile0_h;   // first tile per unit, nunits + 1
    std::vector<int32_t> unit0_h;        // first unit per system, nsys + 1
    std::vector<int32_t> sys_of_unit_h;  // nunits
    // device
    int32_t *rowptr, *colind, *sys_of_tile, *cta0;
    int32_t *unit_tile0, *unit0, *sys_of_unit;
    double* v64;
    float* v32;
    int rows_per_cta = 256;
};

// Rows per CTA of the FP32 root-step kernel, chosen by timing; cached per
// batch shape.
std::mutex g_tune_mu;
std::map<std::tuple<int64_t, int64_t, int>, int> g_tune;

template <int NR>
int32_t launch_bstep_f(const Batch& B, const BStep* steps, const BufSet<float>& bs, int rpc,
                       cudaStream_t s, const int32_t* active = nullptr) {
    k_bstep<float, NR><<<(unsigned)(B.N / rpc), rpc, 0, s>>>(B.rowptr, B.colind, B.v32, steps,
                                                             B.sys_of_tile, bs, nullptr, active);
    BCHECK("k_bstep<float>");
    return PPG_OK;
}

template <int NR>
int32_t launch_bstep_d(const Batch& B, const BStep* steps, const BufSet<double>& bs,
                       double* part, cudaStream_t s, const int32_t* active = nullptr) {
    k_bstep<double, NR><<<(unsigned)(B.N / 256), 256, 0, s>>>(B.rowptr, B.colind, B.v64, steps,
                                                              B.sys_of_tile, bs, part, active);
    BCHECK("k_bstep<double>");
    return PPG_OK;
}

struct Work {
    double* V;          // [(m+1) columns][N * NR]
    float* Z;           // [m][N * NR]
    float *fa, *fb, *fc, *v32;
    double* zd;
    double* X;          // packed solution
    double* Bp;         // packed right-hand sides
    double* part;       // partial sums
    int64_t pstr;
    double *h1, *h2, *nrm;   // [(MAXC+2)][nsolve]
    BStep* steps_p;     // [K][nsys] polynomial passes
    BStep* steps_spmv;  // [nsys] plain SpMV (x = zd, o0 = w)
    BStep* steps_resid; // [nsys]
    BStep* steps_build; // [nsys] SpMV for the construction
    BState st;
    GridBar* gbar;      // grid barrier of the persistent launch
    int32_t* cyc;       // cycles the persistent launch ran
};

template <int NR>
int32_t cgs2_batch(const Batch& B, Work& W, int j, double* wcol, int with_self, int64_t ldV,
                   cudaStream_t s, const int32_t* active = nullptr) {
    const int nsolve = B.nsys * NR;
    const int ncol = j + 1;
    const int64_t pstr = W.pstr;
    for (int pass = 0; pass < 2; ++pass) {
        const int self = (pass == 0) ? with_self : 0;
        const int nvals = ncol + self;
        double* h = pass == 0 ? W.h1 : W.h2;
        k_bdot<NR><<<dim3((unsigned)B.nunits, (nvals + BCH - 1) / BCH), 256, 0, s>>>(
            W.V, ldV, ncol, wcol, self, W.part, pstr, B.unit_tile0, B.sys_of_unit, active);
        BCHECK("k_bdot");
        k_bsegsum<<<dim3(B.nsys, (nvals + 7) / 8), 256, 0, s>>>(W.part, pstr, nvals, NR, B.unit0,
                                                                B.nsys, h);
        BCHECK("k_bsegsum");
        k_bsub<NR><<<(unsigned)B.nunits, 256, 0, s>>>(W.V, ldV, ncol, wcol, h, nsolve,
                                                      B.unit_tile0, B.sys_of_unit, pass == 1,
                                                      W.part, active);
        BCHECK("k_bsub");
    }
    k_bsegsum<<<dim3(B.nsys, 1), 256, 0, s>>>(W.part, NR, 1, NR, B.unit0, B.nsys, W.nrm);
    BCHECK("k_bsegsum");
    return PPG_OK;
}

template <int NR>
int32_t tune_rows(Batch& B, Work& W, cudaStream_t s) {
    const auto key = std::make_tuple(B.N, B.nnz, NR);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            B.rows_per_cta = it->second;
            return PPG_OK;
        }
    }
    // time a plain SpMV pass over the batch for each candidate
    std::vector<BStep> hs(B.nsys);
    for (auto& st : hs) st = BStep{OP_SPMV, 0, 0, 0, 0, B_IN, -1, -1, -1, B_A, -1};
    PPG_CUDA(cudaMemcpyAsync(W.steps_spmv, hs.data(), sizeof(BStep) * B.nsys,
                             cudaMemcpyHostToDevice, s));
    BufSet<float> bs{};
    bs.p[B_IN] = W.v32;
    bs.p[B_A] = W.fa;
    PPG_CUDA(cudaMemsetAsync(W.v32, 0, sizeof(float) * B.N * NR, s));
    cudaEvent_t e0, e1;
    PPG_CUDA(cudaEventCreate(&e0));
    PPG_CUDA(cudaEventCreate(&e1));
    int best = 256;
    float best_ms = 1e30f;
    for (int rpc : {64, 128, 256}) {
        PPG_TRY(launch_bstep_f<NR>(B, W.steps_spmv, bs, rpc, s));   // warm-up
        PPG_CUDA(cudaEventRecord(e0, s));
        for (int rep = 0; rep < 3; ++rep) PPG_TRY(launch_bstep_f<NR>(B, W.steps_spmv, bs, rpc, s));
        PPG_CUDA(cudaEventRecord(e1, s));
        PPG_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        PPG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) { best_ms = ms; best = rpc; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B.rows_per_cta = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
    return PPG_OK;
}

// one restart cycle of FGMRES(m) for every solve (no host synchronisation;
// captured as a graph by the caller)
template <int NR>
int32_t cycle_batch(Batch& B, Work& W, int K, double tol, cudaStream_t s) {
    const int nsolve = B.nsys * NR;
    const int64_t ldV = B.N * NR;
    const int64_t total = B.N * NR;
    const int sg = (nsolve + 127) / 128;
    for (int j = 0; j < B.m; ++j) {
        double* w = W.V + (size_t)(j + 1) * ldV;
        float* zj = W.Z + (size_t)j * ldV;
        // (W.v32 = v_j in FP32 was written with the scaling of v_j)
        BufSet<float> fs{};
        fs.p[B_IN] = W.v32;
        fs.p[B_P] = zj;
        fs.p[B_A] = W.fa;
        fs.p[B_B] = W.fb;
        fs.p[B_C] = W.fc;
        for (int k = 0; k < K; ++k)
            PPG_TRY(launch_bstep_f<NR>(B, W.steps_p + (size_t)k * B.nsys, fs, B.rows_per_cta, s,
                                       W.st.active));
        k_cast32<<<elem_grid(total), 256, 0, s>>>(zj, W.zd, total);
        BCHECK("k_cast32");
        BufSet<double> ds{};
        ds.p[B_IN] = W.zd;
        ds.p[B_OUT] = w;
        PPG_TRY(launch_bstep_d<NR>(B, W.steps_spmv, ds, nullptr, s, W.st.active));
        PPG_TRY(cgs2_batch<NR>(B, W, j, w, 0, ldV, s, W.st.active));
        k_bgivens<<<sg, 128, 0, s>>>(W.st, nsolve, B.ldh, B.m, j, W.h1, W.h2, W.nrm, 0, tol);
        BCHECK("k_bgivens");
        k_bscale<NR><<<elem_grid(total), 256, 0, s>>>(w, W.st.inv, B.sys_of_tile, total, W.v32);
        BCHECK("k_bscale");
    }
    k_bbacksolve<<<(unsigned)(((int64_t)nsolve * 32 + 127) / 128), 128, 0, s>>>(W.st, nsolve, B.ldh,
                                                                          B.m);
    BCHECK("k_bbacksolve");
    k_bzy<NR><<<elem_grid(total), 256, 0, s>>>(W.Z, ldV, W.X, W.st, B.sys_of_tile, B.m, total);
    BCHECK("k_bzy");
    BufSet<double> rs{};
    rs.p[B_IN] = W.X;
    rs.p[B_P] = W.Bp;    // a0: b
    rs.p[B_OUT] = W.V;   // r into V_0
    PPG_TRY(launch_bstep_d<NR>(B, W.steps_resid, rs, W.part, s));
    k_bsegsum<<<dim3(B.nsys, 1), 256, 0, s>>>(W.part, NR, 1, NR, B.cta0, B.nsys, W.nrm);
    BCHECK("k_bsegsum");
    k_bcycle<<<sg, 128, 0, s>>>(W.st, nsolve, B.m, W.nrm, tol, 0);
    BCHECK("k_bcycle");
    k_bscale<NR><<<elem_grid(total), 256, 0, s>>>(W.V, W.st.inv, B.sys_of_tile, total, W.v32);
    BCHECK("k_bscale");
    return PPG_OK;
}

// The whole solve as one persistent cooperative launch (captured as a
// one-node CUDA graph on a non-legacy stream).  Returns after the stream
// has synchronised; *cycles_out = restart cycles run.
template <int NR>
int32_t run_persistent(const Batch& B, Work& W, int K, double tol, int max_cycles,
                       double timeout_ms, cudaStream_t s, int* cycles_out) {
    PArgs a{};
    a.rowptr = B.rowptr;
    a.colind = B.colind;
    a.v64 = B.v64;
    a.v32 = B.v32;
    a.sys_of_tile = B.sys_of_tile;
    a.unit_tile0 = B.unit_tile0;
    a.unit0 = B.unit0;
    a.sys_of_unit = B.sys_of_unit;
    a.cta0 = B.cta0;
    a.nsys = B.nsys;
    a.m = B.m;
    a.ldh = B.ldh;
    a.K = K;
    a.max_cycles = max_cycles;
    // FP32 root steps on row groups of 64 rows, four per CTA (whole 64 x 4
    // batching call: 64 rows 1.32 s, 128 rows 1.33 s, 256 rows 1.37 s; the
    // per-cycle graph's tuned kernel prefers 256: 1.22 s against 1.30 s and
    // 1.51 s)
    a.rows = 64;
    a.N = B.N;
    a.nunits = B.nunits;
    a.ntiles = B.ntiles;
    a.tol = tol;
    a.V = W.V;
    a.Z = W.Z;
    a.fa = W.fa;
    a.fb = W.fb;
    a.fc = W.fc;
    a.x32 = W.v32;
    a.zd = W.zd;
    a.X = W.X;
    a.Bp = W.Bp;
    a.part = W.part;
    a.pstr = W.pstr;
    a.h1 = W.h1;
    a.h2 = W.h2;
    a.nrm = W.nrm;
    a.steps_p = W.steps_p;
    a.steps_spmv = W.steps_spmv;
    a.steps_resid = W.steps_resid;
    a.st = W.st;
    a.bar = W.gbar;
    a.timeout_ns = (unsigned long long)(std::max(0.0, timeout_ms) * 1e6);
    a.cycles_out = W.cyc;
    if (a.rows != 64 && a.rows != 128 && a.rows != 256) return PPG_ERR_ARG;
    int occ = 0;
    PPG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bpersist<NR>, 256, 0));
    if (occ < 1) {
        set_cuda_error(cudaErrorInvalidConfiguration, "k_bpersist: no resident CTA");
        return PPG_ERR_CUDA;
    }
    // every CTA resident (cooperative launch); no more CTAs than tiles
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)occ * device_sm_count(), B.ntiles));
    PPG_CUDA(cudaMemsetAsync(W.gbar, 0, sizeof(GridBar), s));
    PPG_CUDA(cudaMemsetAsync(W.cyc, 0, sizeof(int32_t), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    bool launched = false;
    if (s != nullptr) {
        cudaStreamCaptureStatus cs;
        PPG_CUDA(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone) return PPG_ERR_ARG;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t gexec = nullptr;
        PPG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const cudaError_t el = cudaLaunchKernelEx(&cfg, k_bpersist<NR>, a);
        const cudaError_t ee = cudaStreamEndCapture(s, &graph);
        if (el == cudaSuccess && ee == cudaSuccess &&
            cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess) {
            const cudaError_t eg = cudaGraphLaunch(gexec, s);
            const cudaError_t es = cudaStreamSynchronize(s);
            cudaGraphExecDestroy(gexec);
            cudaGraphDestroy(graph);
            if (eg != cudaSuccess) { set_cuda_error(eg, "cudaGraphLaunch(k_bpersist)"); return PPG_ERR_CUDA; }
            if (es != cudaSuccess) { set_cuda_error(es, "k_bpersist"); return PPG_ERR_CUDA; }
            launched = true;
        } else {
            // this runtime cannot capture the cooperative launch: launch it directly
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
        }
    }
    if (!launched) {
        PPG_CUDA(cudaLaunchKernelEx(&cfg, k_bpersist<NR>, a));
        PPG_CUDA(cudaStreamSynchronize(s));
    }
    ++g_launches;
    GridBar gb{};
    int32_t cyc = 0;
    PPG_CUDA(cudaMemcpy(&gb, W.gbar, sizeof(GridBar), cudaMemcpyDeviceToHost));
    PPG_CUDA(cudaMemcpy(&cyc, W.cyc, sizeof(int32_t), cudaMemcpyDeviceToHost));
    *cycles_out = cyc;
    return gb.err ? PPG_ERR_TIMEOUT : PPG_OK;
}

}  // namespace
}  // namespace ppg

using namespace ppg;

template <int NR>
static int32_t solve_batched_impl(int32_t nsys, const ppg_csr* As, const double* const* Bsrc,
                                  double* const* Xdst, const double* const* v0, int32_t d,
                                  int32_t m, double tol, const ppg_opts* o, ppg_roots* roots_out,
                                  ppg_stats* stats, double* relres_out, int32_t* iters_out,
                                  cudaStream_t s) {
    const int64_t launches0 = g_launches;
    Batch B;
    B.nsys = nsys;
    B.NR = NR;
    B.m = m;
    B.d = d;
    const int mk = std::max(m, d);      // Krylov columns for both phases
    B.ldh = mk + 1;
    B.off.resize(nsys);
    B.n.resize(nsys);
    B.tile0_h.resize(nsys + 1);
    int64_t N = 0, nnz = 0;
    for (int i = 0; i < nsys; ++i) {
        B.off[i] = N;
        B.n[i] = As[i].n;
        B.tile0_h[i] = (int32_t)(N / BT);
        N += ((int64_t)As[i].n + BT - 1) / BT * BT;
        nnz += As[i].nnz;
    }
    B.tile0_h[nsys] = (int32_t)(N / BT);
    if (N * NR >= ((int64_t)1 << 31) || nnz >= ((int64_t)1 << 31)) return PPG_ERR_ARG;
    B.N = N;
    B.nnz = nnz;
    B.ntiles = N / BT;
    B.unit_tile0_h.clear();
    B.sys_of_unit_h.clear();
    B.unit0_h.assign(nsys + 1, 0);
    for (int i = 0; i < nsys; ++i) {
        B.unit0_h[i] = (int32_t)B.unit_tile0_h.size();
        for (int32_t t = B.tile0_h[i]; t < B.tile0_h[i + 1]; t += BUNIT) {
            B.unit_tile0_h.push_back(t);
            B.sys_of_unit_h.push_back(i);
        }
    }
    B.unit0_h[nsys] = (int32_t)B.unit_tile0_h.size();
    B.nunits = (int64_t)B.unit_tile0_h.size();
    B.unit_tile0_h.push_back((int32_t)B.ntiles);
    const int nsolve = nsys * NR;
    const int64_t ldV = N * NR;

    // polynomial plans are built after the construction; their length K is
    // bounded by the capacity of the roots
    Arena ar;
    Work W{};
    ar.add(&B.rowptr, (size_t)N + 1);
    ar.add(&B.colind, (size_t)nnz);
    ar.add(&B.v64, (size_t)nnz);
    ar.add(&B.v32, (size_t)nnz);
    ar.add(&B.sys_of_tile, (size_t)B.ntiles);
    ar.add(&B.cta0, (size_t)nsys + 1);
    ar.add(&B.unit_tile0, (size_t)B.nunits + 1);
    ar.add(&B.unit0, (size_t)nsys + 1);
    ar.add(&B.sys_of_unit, (size_t)std::max<int64_t>(B.nunits, 1));
    ar.add(&W.V, (size_t)(mk + 1) * ldV);
    ar.add(&W.Z, (size_t)m * ldV);
    ar.add(&W.fa, (size_t)ldV);
    ar.add(&W.fb, (size_t)ldV);
    ar.add(&W.fc, (size_t)ldV);
    ar.add(&W.v32, (size_t)ldV);
    ar.add(&W.zd, (size_t)ldV);
    ar.add(&W.X, (size_t)ldV);
    ar.add(&W.Bp, (size_t)ldV);
    W.pstr = (int64_t)(ORTHO_MAXC + 2) * NR;
    ar.add(&W.part, (size_t)(B.ntiles + 16) * W.pstr);
    ar.add(&W.h1, (size_t)(ORTHO_MAXC + 2) * nsolve);
    ar.add(&W.h2, (size_t)(ORTHO_MAXC + 2) * nsolve);
    ar.add(&W.nrm, (size_t)nsolve);
    const int Kmax = 4 * d + 8;
    ar.add(&W.steps_p, (size_t)Kmax * nsys);
    ar.add(&W.steps_spmv, (size_t)nsys);
    ar.add(&W.steps_resid, (size_t)nsys);
    ar.add(&W.steps_build, (size_t)nsys);
    ar.add(&W.st.R, (size_t)nsolve * B.ldh * mk);
    ar.add(&W.st.Hraw, (size_t)nsys * B.ldh * mk);
    ar.add(&W.st.cs, (size_t)nsolve * mk);
    ar.add(&W.st.sn, (size_t)nsolve * mk);
    ar.add(&W.st.g, (size_t)nsolve * (mk + 1));
    ar.add(&W.st.y, (size_t)nsolve * mk);
    ar.add(&W.st.inv, (size_t)nsolve);
    ar.add(&W.st.bnorm, (size_t)nsolve);
    ar.add(&W.st.relres, (size_t)nsolve);
    ar.add(&W.st.active, (size_t)nsolve);
    ar.add(&W.st.ksteps, (size_t)nsolve);
    ar.add(&W.st.iters, (size_t)nsolve);
    ar.add(&W.st.brk, (size_t)nsolve);
    ar.add(&W.gbar, 1);
    ar.add(&W.cyc, 1);
    PPG_TRY(ar.alloc(s));
    struct Guard { Arena& a; cudaStream_t s; ~Guard() { a.release(s); } } guard{ar, s};

    // ---- pack ----
    std::vector<int32_t> sot(B.ntiles);
    for (int i = 0; i < nsys; ++i)
        for (int t = B.tile0_h[i]; t < B.tile0_h[i + 1]; ++t) sot[t] = i;
    PPG_CUDA(cudaMemcpyAsync(B.sys_of_tile, sot.data(), sizeof(int32_t) * B.ntiles,
                             cudaMemcpyHostToDevice, s));
    PPG_CUDA(cudaMemcpyAsync(B.unit_tile0, B.unit_tile0_h.data(),
                             sizeof(int32_t) * (B.nunits + 1), cudaMemcpyHostToDevice, s));
    PPG_CUDA(cudaMemcpyAsync(B.unit0, B.unit0_h.data(), sizeof(int32_t) * (nsys + 1),
                             cudaMemcpyHostToDevice, s));
    if (B.nunits > 0)
        PPG_CUDA(cudaMemcpyAsync(B.sys_of_unit, B.sys_of_unit_h.data(),
                                 sizeof(int32_t) * B.nunits, cudaMemcpyHostToDevice, s));
    int64_t nz_off = 0;
    for (int i = 0; i < nsys; ++i) {
        const int32_t np = B.tile0_h[i + 1] * BT - B.tile0_h[i] * BT;
        k_pack_csr<<<elem_grid(std::max<int64_t>(np, As[i].nnz)), 256, 0, s>>>(
            As[i].rowptr, As[i].colind, (const double*)As[i].vals, As[i].n, np, B.off[i], nz_off,
            B.rowptr, B.colind, B.v64, B.v32);
        BCHECK("k_pack_csr");
        nz_off += As[i].nnz;
    }
    {
        const int32_t last = (int32_t)nnz;
        PPG_CUDA(cudaMemcpyAsync(B.rowptr + N, &last, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    // stopped systems skip their rows, so basis columns they never write
    // must hold finite values: start from zeros
    PPG_CUDA(cudaMemsetAsync(W.V, 0, sizeof(double) * (size_t)(mk + 1) * ldV, s));
    PPG_CUDA(cudaMemsetAsync(W.Z, 0, sizeof(float) * (size_t)m * ldV, s));
    PPG_CUDA(cudaMemsetAsync(W.st.R, 0, sizeof(double) * nsolve * B.ldh * mk, s));
    PPG_CUDA(cudaMemsetAsync(W.st.Hraw, 0, sizeof(double) * nsys * B.ldh * mk, s));
    PPG_CUDA(cudaMemsetAsync(W.st.iters, 0, sizeof(int32_t) * nsolve, s));
    const int sg1 = (nsys + 127) / 128;
    const int sgn = (nsolve + 127) / 128;

    // ---- construction: one GMRES(d) for every system (one rhs slot) ----
    std::vector<ppg_roots> roots(nsys);
    std::vector<std::vector<double>> rre(nsys), rim(nsys);
    {
        for (int i = 0; i < nsys; ++i) {
            const int32_t np = B.tile0_h[i + 1] * BT - B.tile0_h[i] * BT;
            k_pack_vec<<<elem_grid(np), 256, 0, s>>>(v0[i], As[i].n, np, 1, B.off[i], W.V, 1);
            BCHECK("k_pack_vec");
        }
        // ||v0|| per system, V_0 = v0 / ||v0||
        k_bdot<1><<<dim3((unsigned)B.nunits, 1), 256, 0, s>>>(W.V, N, 0, W.V, 1, W.part, W.pstr,
                                                               B.unit_tile0, B.sys_of_unit,
                                                               nullptr);
        BCHECK("k_bdot");
        k_bsegsum<<<dim3(nsys, 1), 256, 0, s>>>(W.part, W.pstr, 1, 1, B.unit0, nsys, W.nrm);
        BCHECK("k_bsegsum");
        BState bst = W.st;
        PPG_CUDA(cudaMemsetAsync(bst.brk, 0xff, sizeof(int32_t) * nsys, s));
        k_bcycle<<<sg1, 128, 0, s>>>(bst, nsys, mk, W.nrm, -1.0, 1);   // inv = 1/||v0||
        BCHECK("k_bcycle");
        k_bscale<1><<<elem_grid(N), 256, 0, s>>>(W.V, bst.inv, B.sys_of_tile, N, nullptr);
        BCHECK("k_bscale");
        std::vector<BStep> hs(nsys);
        for (auto& st : hs) st = BStep{OP_SPMV, 0, 0, 0, 0, B_IN, -1, -1, -1, B_OUT, -1};
        PPG_CUDA(cudaMemcpyAsync(W.steps_build, hs.data(), sizeof(BStep) * nsys,
                                 cudaMemcpyHostToDevice, s));
        for (int j = 0; j < d; ++j) {
            double* vj = W.V + (size_t)j * N;
            double* w = W.V + (size_t)(j + 1) * N;
            BufSet<double> ds{};
            ds.p[B_IN] = vj;
            ds.p[B_OUT] = w;
            PPG_TRY(launch_bstep_d<1>(B, W.steps_build, ds, nullptr, s));
            PPG_TRY(cgs2_batch<1>(B, W, j, w, 1, N, s));
            k_bgivens<<<sg1, 128, 0, s>>>(bst, nsys, B.ldh, mk, j, W.h1, W.h2, W.nrm, 1, 0.0);
            BCHECK("k_bgivens");
            k_bscale<1><<<elem_grid(N), 256, 0, s>>>(w, bst.inv, B.sys_of_tile, N, nullptr);
            BCHECK("k_bscale");
        }
        std::vector<double> H((size_t)nsys * B.ldh * mk);
        std::vector<int32_t> brk(nsys);
        PPG_CUDA(cudaMemcpyAsync(H.data(), W.st.Hraw, sizeof(double) * H.size(),
                                 cudaMemcpyDeviceToHost, s));
        PPG_CUDA(cudaMemcpyAsync(brk.data(), W.st.brk, sizeof(int32_t) * nsys,
                                 cudaMemcpyDeviceToHost, s));
        PPG_CUDA(cudaStreamSynchronize(s));
        ppg_opts ro = *o;
        for (int i = 0; i < nsys; ++i) {
            const int d_eff = brk[i] >= 0 ? brk[i] + 1 : d;
            const int cap = 4 * d + 8;
            rre[i].assign(cap, 0.0);
            rim[i].assign(cap, 0.0);
            roots[i] = ppg_roots{0, 0, 0, cap, rre[i].data(), rim[i].data(), nullptr};
            int32_t rc = ppg_roots_from_hessenberg(H.data() + (size_t)i * B.ldh * mk, B.ldh,
                                                   d_eff, &ro, &roots[i]);
            if (rc < 0) return rc;
            if (roots_out) {
                ppg_roots& ro_i = roots_out[i];
                if (ro_i.capacity < roots[i].n_total || !ro_i.re || !ro_i.im) return PPG_ERR_CAPACITY;
                ro_i.n_orig = roots[i].n_orig;
                ro_i.n_added = roots[i].n_added;
                ro_i.n_total = roots[i].n_total;
                std::memcpy(ro_i.re, rre[i].data(), sizeof(double) * roots[i].n_total);
                std::memcpy(ro_i.im, rim[i].data(), sizeof(double) * roots[i].n_total);
            }
        }
    }

    // ---- polynomial step table: one column per system, padded with no-ops ----
    std::vector<std::vector<Step>> plans(nsys);
    int K = 0;
    for (int i = 0; i < nsys; ++i) {
        plans[i] = plan_p(roots[i].re, roots[i].im, roots[i].n_total, false);
        K = std::max<int>(K, (int)plans[i].size());
    }
    if (K > Kmax) return PPG_ERR_CAPACITY;
    {
        std::vector<BStep> hs((size_t)K * nsys);
        for (int k = 0; k < K; ++k)
            for (int i = 0; i < nsys; ++i) {
                BStep& b = hs[(size_t)k * nsys + i];
                if (k < (int)plans[i].size()) {
                    const Step& p = plans[i][k];
                    b = BStep{p.op, p.flags, p.c1, p.c2, p.c3, p.x, p.a0, p.a1, p.a2, p.o0, p.o1};
                } else {
                    b = BStep{OP_NOP, 0, 0, 0, 0, -1, -1, -1, -1, -1, -1};
                }
            }
        PPG_CUDA(cudaMemcpyAsync(W.steps_p, hs.data(), sizeof(BStep) * hs.size(),
                                 cudaMemcpyHostToDevice, s));
        std::vector<BStep> sp(nsys), rs(nsys);
        for (int i = 0; i < nsys; ++i) {
            sp[i] = BStep{OP_SPMV, 0, 0, 0, 0, B_IN, -1, -1, -1, B_OUT, -1};
            rs[i] = BStep{OP_RESID, 0, 0, 0, 0, B_IN, B_P, -1, -1, B_OUT, -1};
        }
        PPG_CUDA(cudaMemcpyAsync(W.steps_resid, rs.data(), sizeof(BStep) * nsys,
                                 cudaMemcpyHostToDevice, s));
        // the tuner overwrites steps_spmv; set the solve's table after it
        PPG_TRY(tune_rows<NR>(B, W, s));
        PPG_CUDA(cudaMemcpyAsync(W.steps_spmv, sp.data(), sizeof(BStep) * nsys,
                                 cudaMemcpyHostToDevice, s));
    }
    // per-system CTA ranges of the residual kernel (256 rows per CTA)
    PPG_CUDA(cudaMemcpyAsync(B.cta0, B.tile0_h.data(), sizeof(int32_t) * (nsys + 1),
                             cudaMemcpyHostToDevice, s));

    // ---- solve: x = 0, r = b ----
    for (int i = 0; i < nsys; ++i) {
        const int32_t np = B.tile0_h[i + 1] * BT - B.tile0_h[i] * BT;
        k_pack_vec<<<elem_grid((int64_t)np * NR), 256, 0, s>>>(Bsrc[i], As[i].n, np, NR, B.off[i],
                                                              W.Bp, NR);
        BCHECK("k_pack_vec");
    }
    PPG_CUDA(cudaMemsetAsync(W.X, 0, sizeof(double) * ldV, s));
    PPG_CUDA(cudaMemcpyAsync(W.V, W.Bp, sizeof(double) * ldV, cudaMemcpyDeviceToDevice, s));
    k_bdot<NR><<<dim3((unsigned)B.nunits, 1), 256, 0, s>>>(W.V, ldV, 0, W.V, 1, W.part, W.pstr,
                                                           B.unit_tile0, B.sys_of_unit, nullptr);
    BCHECK("k_bdot");
    k_bsegsum<<<dim3(nsys, 1), 256, 0, s>>>(W.part, W.pstr, 1, NR, B.unit0, nsys, W.nrm);
    BCHECK("k_bsegsum");
    k_bcycle<<<sgn, 128, 0, s>>>(W.st, nsolve, m, W.nrm, tol, 1);
    BCHECK("k_bcycle");
    k_bscale<NR><<<elem_grid(ldV), 256, 0, s>>>(W.V, W.st.inv, B.sys_of_tile, ldV, W.v32);
    BCHECK("k_bscale");
    // the Krylov state of the solve uses m columns
    Batch Bs = B;
    Bs.m = m;
    Bs.ldh = m + 1;

    std::vector<double> rel(nsolve);
    std::vector<int32_t> act(nsolve);
    const int max_cycles = o->max_cycles > 0 ? o->max_cycles : 10000;
    int cycles = 0;
    bool all = false;
    if (o->batch_mode == 0) {
        // every cycle of every solve in one persistent launch
        PPG_TRY(run_persistent<NR>(Bs, W, K, tol, max_cycles, o->wait_timeout_ms, s, &cycles));
        PPG_CUDA(cudaMemcpyAsync(rel.data(), W.st.relres, sizeof(double) * nsolve,
                                 cudaMemcpyDeviceToHost, s));
        PPG_CUDA(cudaMemcpyAsync(act.data(), W.st.active, sizeof(int32_t) * nsolve,
                                 cudaMemcpyDeviceToHost, s));
        PPG_CUDA(cudaStreamSynchronize(s));
        all = true;
        for (int i = 0; i < nsolve; ++i) {
            if (!std::isfinite(rel[i])) return PPG_ERR_NONFINITE;
            if (act[i]) all = false;
        }
    } else {
        // capture one restart cycle as a graph (not possible on the legacy
        // default stream: there the cycle is launched directly)
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t gexec = nullptr;
        int64_t launches_per_cycle = 0;
        if (s != nullptr) {
            cudaStreamCaptureStatus cs;
            PPG_CUDA(cudaStreamIsCapturing(s, &cs));
            if (cs != cudaStreamCaptureStatusNone) return PPG_ERR_ARG;
            PPG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            const int64_t l0 = g_launches;
            int32_t rc = cycle_batch<NR>(Bs, W, K, tol, s);
            const int64_t per_cycle = g_launches - l0;
            g_launches = l0;
            cudaError_t e = cudaStreamEndCapture(s, &graph);
            if (rc < 0) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) {
                set_cuda_error(e, "cudaStreamEndCapture");
                return PPG_ERR_CUDA;
            }
            e = cudaGraphInstantiate(&gexec, graph, 0);
            if (e != cudaSuccess) {
                cudaGraphDestroy(graph);
                set_cuda_error(e, "cudaGraphInstantiate");
                return PPG_ERR_CUDA;
            }
            launches_per_cycle = per_cycle;
        }
        struct GGuard {
            cudaGraph_t g;
            cudaGraphExec_t x;
            ~GGuard() {
                if (x) cudaGraphExecDestroy(x);
                if (g) cudaGraphDestroy(g);
            }
        } gg{graph, gexec};
        while (cycles < max_cycles) {
            if (gexec) {
                PPG_CUDA(cudaGraphLaunch(gexec, s));
                g_launches += launches_per_cycle;
            } else {
                PPG_TRY(cycle_batch<NR>(Bs, W, K, tol, s));
            }
            ++cycles;
            PPG_CUDA(cudaMemcpyAsync(rel.data(), W.st.relres, sizeof(double) * nsolve,
                                     cudaMemcpyDeviceToHost, s));
            PPG_CUDA(cudaMemcpyAsync(act.data(), W.st.active, sizeof(int32_t) * nsolve,
                                     cudaMemcpyDeviceToHost, s));
            PPG_CUDA(cudaStreamSynchronize(s));
            all = true;
            for (int i = 0; i < nsolve; ++i) {
                if (!std::isfinite(rel[i])) return PPG_ERR_NONFINITE;
                if (act[i]) all = false;
            }
            if (all) break;
        }
    }
    // ---- unpack ----
    for (int i = 0; i < nsys; ++i) {
        k_unpack_vec<<<elem_grid((int64_t)As[i].n * NR), 256, 0, s>>>(W.X, As[i].n, NR, B.off[i],
                                                                     Xdst[i], NR);
        BCHECK("k_unpack_vec");
    }
    std::vector<int32_t> its(nsolve);
    PPG_CUDA(cudaMemcpyAsync(its.data(), W.st.iters, sizeof(int32_t) * nsolve,
                             cudaMemcpyDeviceToHost, s));
    PPG_CUDA(cudaStreamSynchronize(s));
    if (relres_out) std::memcpy(relres_out, rel.data(), sizeof(double) * nsolve);
    if (iters_out) std::memcpy(iters_out, its.data(), sizeof(int32_t) * nsolve);
    if (stats) {
        *stats = ppg_stats{};
        int64_t it = 0;
        double worst = 0.0;
        for (int i = 0; i < nsolve; ++i) {
            it += its[i];
            worst = std::max(worst, rel[i]);
        }
        stats->iters = it;
        stats->cycles = cycles;
        stats->true_relres = worst;
        stats->converged = all ? 1 : 0;
        stats->launches = g_launches - launches0;
    }
    return all ? PPG_OK : PPG_NOT_CONVERGED;
}

extern "C" int32_t ppg_solve_batched(int32_t nsys, const ppg_csr* As, int32_t nrhs,
                                     const double* const* B, double* const* X,
                                     const double* const* v0, int32_t d, int32_t m, double tol,
                                     const ppg_opts* opts, ppg_roots* roots_out,
                                     ppg_stats* stats, double* relres_out, int32_t* iters_out,
                                     void* stream) {
    if (nsys < 1 || !As || !B || !X || !v0 || (nrhs != 1 && nrhs != 4)) return PPG_ERR_ARG;
    if (d < 1 || m < 1 || m + 1 > ORTHO_MAXC || d + 1 > ORTHO_MAXC || !(tol > 0.0))
        return PPG_ERR_ARG;
    for (int i = 0; i < nsys; ++i) {
        const ppg_csr& A = As[i];
        if (A.n < 1 || A.nnz < 0 || !A.rowptr || (A.nnz > 0 && (!A.colind || !A.vals)) ||
            A.dtype != PPG_F64 || !B[i] || !X[i] || !v0[i])
            return PPG_ERR_ARG;
    }
    ppg_opts o;
    ppg_default_opts(&o);
    if (opts) o = *opts;
    PPG_CUDA(cudaGetLastError());
    cudaStream_t s = (cudaStream_t)stream;
    if (nrhs == 4)
        return solve_batched_impl<4>(nsys, As, B, X, v0, d, m, tol, &o, roots_out, stats,
                                     relres_out, iters_out, s);
    return solve_batched_impl<1>(nsys, As, B, X, v0, d, m, tol, &o, roots_out, stats, relres_out,
                                 iters_out, s);
}
