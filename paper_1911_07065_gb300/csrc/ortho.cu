// Orthogonalisation (CGS2) and the small dense steps of GMRES: Givens
// least squares (Section 3.2 shortcut residual), back substitution, the
// solution update V y, norms and scaling.
//
// The basis V is column-major with leading dimension ldv (>= n, padded so
// each column starts on a 512-byte boundary).  CGS2 runs as three passes
// over the active columns:
//   pass 1  h1 = V^T w                          (k_cgs<0>)
//   pass 2  w -= V h1, then h2 = V^T w          (k_cgs<1>)
//   pass 3  w -= V h2, then ||w||^2             (k_cgs<2>)
// Passes 2 and 3 stage a tile of ORTHO_TR rows x ncol columns of V in
// shared memory, so the column sums and the dot products of the same tile
// read V from HBM once.  Each pass ends with a deterministic reduction of
// the per-CTA partial sums done by the last CTA to finish (no extra
// launch; the counter resets itself).
#include "ppg_common.cuh"

namespace ppg {

constexpr int ORTHO_THREADS = 256;
constexpr int ORTHO_TR = 32;                          // rows per tile
constexpr int ORTHO_WARPS = ORTHO_THREADS / 32;

int ortho_grid(int32_t n) {
    int tiles = (n + ORTHO_TR - 1) / ORTHO_TR;
    return max(1, min(tiles, 152 * 4));
}

size_t ortho_part_doubles(int grid) { return (size_t)grid * (ORTHO_MAXC + 2); }

__device__ __forceinline__ double warp_sum(double v) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

// Reduce part[b * stride + c] over b for c < nvals, in block order; result
// to out[c].  Called by every thread of the last CTA.
__device__ void final_reduce(const double* part, int nblocks, int stride, int nvals,
                             double* out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = warp; c < nvals; c += ORTHO_WARPS) {
        double s = 0.0;
        for (int b = lane; b < nblocks; b += 32) s += __ldcg(part + (size_t)b * stride + c);
        s = warp_sum(s);
        if (lane == 0) out[c] = s;
    }
}

// MODE 0: dots of w with ncol columns (+ w.w if with_self)
// MODE 1: w -= V hin ; dots of the new w with ncol columns
// MODE 2: w -= V hin ; ||w||^2
// Warp wp accumulates columns wp, wp + 8, ...: at most CPW of them, so
// ncol <= 8 * CPW.
template <int MODE, int ORTHO_CPW>
__global__ void __launch_bounds__(ORTHO_THREADS)
k_cgs(const double* __restrict__ V, int64_t ldv, int ncol, double* w, int32_t n,
      const double* __restrict__ hin, int with_self, double* part, unsigned* counter,
      double* hout) {
    // shared layout (doubles): sV [tilecols][ORTHO_TR] | sw [ORTHO_TR] |
    // sh [ORTHO_MAXC] | sred [ORTHO_WARPS][ORTHO_TR]; MODE 0 stages no V tile
    extern __shared__ double smem[];
    const int tilecols = (MODE == 0) ? 0 : ncol;
    double* sV = smem;
    double* sw = sV + (size_t)tilecols * ORTHO_TR;
    double* sh = sw + ORTHO_TR;
    double* sred = sh + ORTHO_MAXC;
    __shared__ bool am_last;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (MODE != 0)
        for (int c = tid; c < ncol; c += ORTHO_THREADS) sh[c] = hin[c];

    double acc[ORTHO_CPW];
#pragma unroll
    for (int q = 0; q < ORTHO_CPW; ++q) acc[q] = 0.0;
    double accself = 0.0;

    const int64_t ntiles = ((int64_t)n + ORTHO_TR - 1) / ORTHO_TR;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t r0 = t * ORTHO_TR;
        const int rows = (int)(((int64_t)n - r0) < ORTHO_TR ? ((int64_t)n - r0) : ORTHO_TR);
        __syncthreads();
        if (MODE == 0) {
            // w tile only; V is read straight from global below
            if (tid < ORTHO_TR) sw[tid] = (tid < rows) ? w[r0 + tid] : 0.0;
            __syncthreads();
            const double wv = sw[lane];
#pragma unroll
            for (int q = 0; q < ORTHO_CPW; ++q) {
                const int c = warp + q * ORTHO_WARPS;
                if (c < ncol && lane < rows) acc[q] += __ldcs(V + c * ldv + r0 + lane) * wv;
            }
            if (with_self && warp == 0) accself += wv * wv;
        } else {
            for (int e = tid; e < ncol * ORTHO_TR; e += ORTHO_THREADS) {
                const int c = e / ORTHO_TR, i = e % ORTHO_TR;
                sV[e] = (i < rows) ? __ldcs(V + c * ldv + r0 + i) : 0.0;
            }
            if (tid < ORTHO_TR) sw[tid] = (tid < rows) ? w[r0 + tid] : 0.0;
            __syncthreads();
            // s_i = sum_c V[c][i] hin[c]: warp wp takes columns c = wp (mod 8)
            double s = 0.0;
            for (int c = warp; c < ncol; c += ORTHO_WARPS) s += sV[c * ORTHO_TR + lane] * sh[c];
            sred[warp * ORTHO_TR + lane] = s;
            __syncthreads();
            if (tid < ORTHO_TR) {
                double tot = 0.0;
#pragma unroll
                for (int k = 0; k < ORTHO_WARPS; ++k) tot += sred[k * ORTHO_TR + tid];
                const double nw = sw[tid] - tot;
                sw[tid] = nw;
                if (tid < rows) w[r0 + tid] = nw;
            }
            __syncthreads();
            const double wv = sw[lane];
            if (MODE == 1) {
#pragma unroll
                for (int q = 0; q < ORTHO_CPW; ++q) {
                    const int c = warp + q * ORTHO_WARPS;
                    if (c < ncol) acc[q] += sV[c * ORTHO_TR + lane] * wv;
                }
            } else if (warp == 0) {
                accself += wv * wv;
            }
        }
    }

    // per-CTA partials: part[blockIdx.x * stride + c]
    const int stride = ORTHO_MAXC + 2;
    double* mypart = part + (size_t)blockIdx.x * stride;
    if (MODE != 2) {
#pragma unroll
        for (int q = 0; q < ORTHO_CPW; ++q) {
            const int c = warp + q * ORTHO_WARPS;
            const double v = warp_sum(acc[q]);
            if (c < ncol && lane == 0) mypart[c] = v;
        }
    }
    const int nvals = (MODE == 2) ? 1 : ncol + ((MODE == 0 && with_self) ? 1 : 0);
    if (MODE == 2 || (MODE == 0 && with_self)) {
        const double v = warp_sum(accself);
        if (warp == 0 && lane == 0) mypart[(MODE == 2) ? 0 : ncol] = v;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (am_last) {
        __threadfence();
        final_reduce(part, gridDim.x, stride, nvals, hout);
        if (tid == 0) *counter = 0u;
    }
}

// dynamic shared bytes for a launch staging `tilecols` columns of V (the
// kernel's layout above; MODE 0 passes 0)
static size_t cgs_smem(int tilecols) {
    return sizeof(double) * ((size_t)tilecols * ORTHO_TR + ORTHO_TR + ORTHO_MAXC +
                             ORTHO_WARPS * ORTHO_TR);
}

static int32_t set_smem_attrs() {
    static bool done = false;   // per process; the attribute is per function
    if (done) return PPG_OK;
    const int mx = (int)cgs_smem(ORTHO_MAXC);
    PPG_CUDA(cudaFuncSetAttribute(k_cgs<1, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    PPG_CUDA(cudaFuncSetAttribute(k_cgs<2, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    PPG_CUDA(cudaFuncSetAttribute(k_cgs<1, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    PPG_CUDA(cudaFuncSetAttribute(k_cgs<2, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    done = true;
    return PPG_OK;
}

int32_t launch_cgs_dot(const double* V, int64_t ldv, int ncol, const double* w,
                       int32_t n, bool with_self, double* h_out, const OrthoWs& ws,
                       cudaStream_t s) {
    if (ncol < 1 || ncol > ORTHO_MAXC) return PPG_ERR_ARG;
    PPG_TRY(set_smem_attrs());
    if (ncol + 1 <= 8 * 8)
        k_cgs<0, 8><<<ws.grid, ORTHO_THREADS, cgs_smem(0), s>>>(
            V, ldv, ncol, const_cast<double*>(w), n, nullptr, with_self ? 1 : 0, ws.part,
            ws.counter, h_out);
    else
        k_cgs<0, 32><<<ws.grid, ORTHO_THREADS, cgs_smem(0), s>>>(
            V, ldv, ncol, const_cast<double*>(w), n, nullptr, with_self ? 1 : 0, ws.part,
            ws.counter, h_out);
    ++g_launches;
    return check_launch("k_cgs<0>");
}

int32_t launch_cgs_update(const double* V, int64_t ldv, int ncol, double* w, int32_t n,
                          const double* hin, int mode, double* h_out, const OrthoWs& ws,
                          cudaStream_t s) {
    if (ncol < 1 || ncol > ORTHO_MAXC) return PPG_ERR_ARG;
    PPG_TRY(set_smem_attrs());
    const bool small = ncol <= 8 * 8;
    if (mode == 1 && small)
        k_cgs<1, 8><<<ws.grid, ORTHO_THREADS, cgs_smem(ncol), s>>>(
            V, ldv, ncol, w, n, hin, 0, ws.part, ws.counter + 1, h_out);
    else if (mode == 1)
        k_cgs<1, 32><<<ws.grid, ORTHO_THREADS, cgs_smem(ncol), s>>>(
            V, ldv, ncol, w, n, hin, 0, ws.part, ws.counter + 1, h_out);
    else if (small)
        k_cgs<2, 8><<<ws.grid, ORTHO_THREADS, cgs_smem(ncol), s>>>(
            V, ldv, ncol, w, n, hin, 0, ws.part, ws.counter + 2, h_out);
    else
        k_cgs<2, 32><<<ws.grid, ORTHO_THREADS, cgs_smem(ncol), s>>>(
            V, ldv, ncol, w, n, hin, 0, ws.part, ws.counter + 2, h_out);
    ++g_launches;
    return check_launch("k_cgs<1/2>");
}

// ---------------------------------------------------------------------------
// Hessenberg column, Givens rotation, shortcut residual (one thread)
// ---------------------------------------------------------------------------

__global__ void k_finish_column(GmresState st, int ldh, int j, const double* h1,
                                const double* h2, const double* nrm, int givens,
                                double bnorm, double brtol) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double* sc = st.scal;
    const double hn = sqrt(fmax(nrm[0], 0.0));
    double col[ORTHO_MAXC + 1];
    for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
    col[j + 1] = hn;
    if (st.Hraw)
        for (int i = 0; i <= j + 1; ++i) st.Hraw[(size_t)j * ldh + i] = col[i];
    bool brk = false;
    if (brtol > 0.0) {
        const double w0 = sqrt(fmax(h1[j + 1], 0.0));   // ||A v_j|| from pass 1
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
        for (int i = 0; i < j; ++i) {
            const double t = st.cs[i] * col[i] + st.sn[i] * col[i + 1];
            col[i + 1] = -st.sn[i] * col[i] + st.cs[i] * col[i + 1];
            col[i] = t;
        }
        const double a = col[j], b = col[j + 1];
        const double r = hypot(a, b);
        double c = 1.0, s = 0.0;
        if (r != 0.0) { c = a / r; s = b / r; }
        st.cs[j] = c;
        st.sn[j] = s;
        col[j] = r;
        col[j + 1] = 0.0;
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
    k_finish_column<<<1, 32, 0, s>>>(st, ldh, j, h1, h2, nrm, givens ? 1 : 0, bnorm, brtol);
    ++g_launches;
    return check_launch("k_finish_column");
}

// y = R^{-1} g (k x k upper triangular), one thread
__global__ void k_backsolve(GmresState st, int ldh, int k) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double s = st.g[i];
        for (int c = i + 1; c < k; ++c) s -= st.R[(size_t)c * ldh + i] * st.y[c];
        st.y[i] = s / st.R[(size_t)i * ldh + i];
    }
}

int32_t launch_backsolve(const GmresState& st, int ldh, int k, cudaStream_t s) {
    k_backsolve<<<1, 32, 0, s>>>(st, ldh, k);
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
    const int grid = max(1, min((n + 255) / 256, 152 * 8));
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
    const double a = *sp;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        y[r] = x[r] * a;
}

int32_t launch_scale(const double* x, double* y, int32_t n, const double* sp,
                     cudaStream_t s) {
    const int grid = max(1, min((n + 255) / 256, 152 * 8));
    k_scale<<<grid, 256, 0, s>>>(x, y, n, sp);
    ++g_launches;
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
    const int grid = max(1, min((n + 255) / 256, 152 * 4));
    k_norm2_part<false><<<grid, 256, 0, s>>>(x, nullptr, n, part);
    ++g_launches;
    *nparts = grid;
    return check_launch("k_norm2_part");
}

int32_t launch_diff_norm2_part(const double* a, const double* b, int32_t n, double* part,
                               cudaStream_t s, int* nparts) {
    const int grid = max(1, min((n + 255) / 256, 152 * 4));
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
    const int grid = max(1, min((n + 255) / 256, 152 * 8));
    k_cast_f64_f32<<<grid, 256, 0, s>>>(x, y, n);
    ++g_launches;
    return check_launch("k_cast_f64_f32");
}
int32_t launch_cast_f32_f64(const float* x, double* y, int32_t n, cudaStream_t s) {
    const int grid = max(1, min((n + 255) / 256, 152 * 8));
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
    const int grid = max(1, min((n + 255) / 256, 152 * 8));
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
    const int grid = max(1, min((n + 255) / 256, 152 * 8));
    k_axpby<T><<<grid, 256, 0, s>>>(a, x, b, y, out, n);
    ++g_launches;
    return check_launch("k_axpby");
}
template int32_t launch_axpby<double>(double, const double*, double, const double*,
                                      double*, int32_t, cudaStream_t);
template int32_t launch_axpby<float>(float, const float*, float, const float*, float*,
                                     int32_t, cudaStream_t);

}  // namespace ppg
