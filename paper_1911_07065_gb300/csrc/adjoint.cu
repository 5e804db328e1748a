// Transposed CSR (for the adjoint solve with A^T) and the adjoint gradient
// on the sparsity pattern.  For x = A^{-1} b and a loss L(x), the adjoint
// lambda = A^{-T} dL/dx gives dL/db = lambda and dL/dA_ij = -lambda_i x_j;
// since p(A^T) = p(A)^T, the adjoint solve reuses the roots of A.
#include "ppg_common.cuh"

namespace ppg {

__global__ void k_count_cols(const int32_t* __restrict__ colind, int32_t nnz,
                             int32_t* cnt) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + colind[k], 1);
}

// out[i] = sum_{j <= i} in[i] for i < N, one CTA of 1024 threads: each
// thread scans a contiguous chunk, the chunk totals are scanned in shared
// memory, then each thread writes its chunk.
__global__ void k_scan_single(const int32_t* in, int32_t* out, int32_t N) {
    __shared__ int32_t ssum[1024];
    const int t = threadIdx.x;
    const int64_t chunk = ((int64_t)N + 1023) / 1024;
    const int64_t lo = t * chunk;
    const int64_t hi = ((int64_t)N < lo + chunk ? (int64_t)N : lo + chunk);
    int32_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += in[i];
    ssum[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int32_t v = (t >= off) ? ssum[t - off] : 0;
        __syncthreads();
        ssum[t] += v;
        __syncthreads();
    }
    int32_t base = (t > 0) ? ssum[t - 1] : 0;
    for (int64_t i = lo; i < hi; ++i) {
        base += in[i];
        out[i] = base;
    }
}

template <typename T>
__global__ void k_scatter_t(const int32_t* __restrict__ rowptr,
                            const int32_t* __restrict__ colind, const T* __restrict__ vals,
                            int32_t n, int32_t* cursor, int32_t* colind_t, T* vals_t,
                            int32_t* perm) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const int32_t pos = atomicAdd(cursor + colind[k], 1);
            colind_t[pos] = (int32_t)i;
            vals_t[pos] = vals[k];
            if (perm) perm[pos] = k;
        }
    }
}

// sort each row of A^T by column (insertion sort; the atomics above leave
// the order within a row arbitrary, the keys are distinct)
template <typename T>
__global__ void k_sort_rows(const int32_t* __restrict__ rowptr_t, int32_t n,
                            int32_t* colind_t, T* vals_t, int32_t* perm) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t lo = rowptr_t[j], hi = rowptr_t[j + 1];
        for (int32_t a = lo + 1; a < hi; ++a) {
            const int32_t key = colind_t[a];
            const T v = vals_t[a];
            const int32_t pk = perm ? perm[a] : 0;
            int32_t b = a - 1;
            while (b >= lo && colind_t[b] > key) {
                colind_t[b + 1] = colind_t[b];
                vals_t[b + 1] = vals_t[b];
                if (perm) perm[b + 1] = perm[b];
                --b;
            }
            colind_t[b + 1] = key;
            vals_t[b + 1] = v;
            if (perm) perm[b + 1] = pk;
        }
    }
}

// work: 2n + 1 int32 of scratch
int32_t launch_transpose(const ppg_csr* A, int32_t* rowptr_t, int32_t* colind_t,
                         void* vals_t, int32_t* perm, int32_t* work, cudaStream_t s) {
    const int32_t n = A->n, nnz = A->nnz;
    int32_t* cnt = work;            // [n]
    int32_t* cursor = work + n;     // [n]
    PPG_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)n, s));
    PPG_CUDA(cudaMemsetAsync(rowptr_t, 0, sizeof(int32_t), s));
    const int gz = max(1, min((nnz + 255) / 256, grid_cap(8)));
    const int gn = max(1, min((n + 255) / 256, grid_cap(8)));
    if (nnz > 0) {
        k_count_cols<<<gz, 256, 0, s>>>(A->colind, nnz, cnt);
        ++g_launches;
        PPG_TRY(check_launch("k_count_cols"));
    }
    k_scan_single<<<1, 1024, 0, s>>>(cnt, rowptr_t + 1, n);
    ++g_launches;
    PPG_TRY(check_launch("k_scan_single"));
    PPG_CUDA(cudaMemcpyAsync(cursor, rowptr_t, sizeof(int32_t) * (size_t)n,
                             cudaMemcpyDeviceToDevice, s));
    if (A->dtype == PPG_F64) {
        k_scatter_t<double><<<gn, 256, 0, s>>>(A->rowptr, A->colind, (const double*)A->vals,
                                               n, cursor, colind_t, (double*)vals_t, perm);
        ++g_launches;
        PPG_TRY(check_launch("k_scatter_t"));
        k_sort_rows<double><<<gn, 256, 0, s>>>(rowptr_t, n, colind_t, (double*)vals_t, perm);
    } else {
        k_scatter_t<float><<<gn, 256, 0, s>>>(A->rowptr, A->colind, (const float*)A->vals,
                                              n, cursor, colind_t, (float*)vals_t, perm);
        ++g_launches;
        PPG_TRY(check_launch("k_scatter_t"));
        k_sort_rows<float><<<gn, 256, 0, s>>>(rowptr_t, n, colind_t, (float*)vals_t, perm);
    }
    ++g_launches;
    return check_launch("k_sort_rows");
}

__global__ void k_adjoint_grad(const int32_t* __restrict__ rowptr,
                               const int32_t* __restrict__ colind,
                               const double* __restrict__ lam, const double* __restrict__ x,
                               int32_t n, double* gvals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double li = lam[i];
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) gvals[k] = -li * x[colind[k]];
    }
}

int32_t launch_adjoint_grad(const ppg_csr* A, const double* lam, const double* x,
                            double* gvals, cudaStream_t s) {
    const int gn = max(1, min((A->n + 255) / 256, grid_cap(8)));
    k_adjoint_grad<<<gn, 256, 0, s>>>(A->rowptr, A->colind, lam, x, A->n, gvals);
    ++g_launches;
    return check_launch("k_adjoint_grad");
}

}  // namespace ppg
