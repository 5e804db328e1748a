// Fused CSR SpMV + root update: one pass over A per root of the GMRES
// polynomial (Algorithm 1: phi(A) v, Algorithm 3: p(A) v), plus the plain
// SpMV and the residual b - A x.
//
// Layout: a CTA owns a tile of SPMV_ROWS consecutive rows.  It stages the
// products vals[k] * x[colind[k]] of the tile's nonzeros in shared memory
// with fully coalesced, streaming loads of vals/colind (consecutive threads
// take consecutive k, so short rows of 5-7 entries cost no idle lanes),
// then thread t sums row t of the tile and applies the root update in the
// epilogue, reading and writing the row-aligned vectors once, coalesced.
// Tiles whose nonzeros exceed the staging buffer are processed in chunks,
// so any row length is handled.
#include "ppg_common.cuh"

namespace ppg {

constexpr int SPMV_ROWS = 256;      // rows per CTA = threads per CTA
constexpr int SPMV_CHUNK_BYTES = 16384;

template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) {
    return __ldcs(p);   // read-once data: evict-first
}

template <typename T, int OP>
__global__ void __launch_bounds__(SPMV_ROWS)
k_spmv_step(const StepArgs<T> a) {
    constexpr int CHUNK = SPMV_CHUNK_BYTES / sizeof(T);
    __shared__ T sprod[CHUNK];
    __shared__ int32_t srp[SPMV_ROWS + 1];
    __shared__ double sred[SPMV_ROWS / 32];

    const int64_t row0 = (int64_t)blockIdx.x * SPMV_ROWS;
    const int tid = threadIdx.x;
    const int nrows = (int)(((int64_t)a.n - row0) < SPMV_ROWS ? ((int64_t)a.n - row0) : SPMV_ROWS);
    for (int i = tid; i <= nrows; i += SPMV_ROWS) srp[i] = __ldg(a.rowptr + row0 + i);
    __syncthreads();
    const int32_t k0 = srp[0];
    const int32_t k1 = srp[nrows];
    const int32_t my_lo = (tid < nrows) ? srp[tid] : k1;
    const int32_t my_hi = (tid < nrows) ? srp[tid + 1] : k1;

    T acc = T(0);
    for (int32_t c0 = k0; c0 < k1; c0 += CHUNK) {
        const int32_t c1 = min(k1, c0 + CHUNK);
#pragma unroll 4
        for (int32_t k = c0 + tid; k < c1; k += SPMV_ROWS) {
            const int32_t col = ld_stream(a.colind + k);
            const T v = ld_stream(a.vals + k);
            sprod[k - c0] = v * __ldg(a.x + col);
        }
        __syncthreads();
        const int32_t lo = max(my_lo, c0);
        const int32_t hi = min(my_hi, c1);
        for (int32_t k = lo; k < hi; ++k) acc += sprod[k - c0];
        __syncthreads();
    }

    double sq = 0.0;
    if (tid < nrows) {
        const int64_t r = row0 + tid;
        const T s = acc;
        if constexpr (OP == OP_SPMV) {
            a.o0[r] = s;
        } else if constexpr (OP == OP_RESID) {
            const T v = __ldg(a.a0 + r) - s;
            a.o0[r] = v;
            sq = (double)v * (double)v;
        } else if constexpr (OP == OP_PHI_REAL) {
            const T pin = __ldg(a.a0 + r) - a.c1 * s;
            a.o0[r] = (a.flags & F_FINAL) ? __ldg(a.a2 + r) - pin : pin;
        } else if constexpr (OP == OP_PHI_PAIR2) {
            const T pin = a.a1[r] + a.c2 * (s - a.c1 * __ldg(a.a0 + r));
            a.o0[r] = (a.flags & F_FINAL) ? __ldg(a.a2 + r) - pin : pin;
        } else if constexpr (OP == OP_P_REAL) {
            const T pr = __ldg(a.a0 + r);
            const T pold = (a.flags & F_PZERO) ? T(0) : a.a1[r];
            const T pnew = pold + a.c1 * pr;
            const T prodn = pr - a.c1 * s;
            if (a.flags & F_FINAL) {
                a.o0[r] = pnew + a.c3 * prodn;
            } else {
                a.o0[r] = pnew;
                a.o1[r] = prodn;
            }
        } else if constexpr (OP == OP_P_PAIR1) {
            const T pr = __ldg(a.a0 + r);
            const T tmp = a.c1 * pr - s;
            const T pold = (a.flags & F_PZERO) ? T(0) : a.a1[r];
            a.o0[r] = pold + a.c2 * tmp;
            if (!(a.flags & F_NO_O1)) a.o1[r] = tmp;
        } else if constexpr (OP == OP_P_PAIR2) {
            const T prodn = __ldg(a.a0 + r) - a.c2 * s;
            if (a.flags & F_FINAL) {
                a.o0[r] = a.a1[r] + a.c3 * prodn;
            } else {
                a.o0[r] = prodn;
            }
        }
    }
    if constexpr (OP == OP_RESID) {
        // deterministic block reduction of ||r||^2
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

int32_t spmv_grid_blocks(int32_t n) { return (n + SPMV_ROWS - 1) / SPMV_ROWS; }

template <typename T>
int32_t launch_step(int op, const StepArgs<T>& a, cudaStream_t s) {
    if (a.n <= 0) return 0;
    const int grid = spmv_grid_blocks(a.n);
    switch (op) {
        case OP_SPMV: k_spmv_step<T, OP_SPMV><<<grid, SPMV_ROWS, 0, s>>>(a); break;
        case OP_RESID: k_spmv_step<T, OP_RESID><<<grid, SPMV_ROWS, 0, s>>>(a); break;
        case OP_PHI_REAL: k_spmv_step<T, OP_PHI_REAL><<<grid, SPMV_ROWS, 0, s>>>(a); break;
        case OP_PHI_PAIR2: k_spmv_step<T, OP_PHI_PAIR2><<<grid, SPMV_ROWS, 0, s>>>(a); break;
        case OP_P_REAL: k_spmv_step<T, OP_P_REAL><<<grid, SPMV_ROWS, 0, s>>>(a); break;
        case OP_P_PAIR1: k_spmv_step<T, OP_P_PAIR1><<<grid, SPMV_ROWS, 0, s>>>(a); break;
        case OP_P_PAIR2: k_spmv_step<T, OP_P_PAIR2><<<grid, SPMV_ROWS, 0, s>>>(a); break;
        default: return PPG_ERR_ARG;
    }
    ++g_launches;
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
