// Dense kernels of the coarsest multigrid level: Gauss-Jordan inversion with
// partial pivoting, the gather / dense matvec / scatter of the coarsest solve,
// and connected components of the active coarsest cells (the scalar Laplacian
// D A D^T has one constant null vector per component; the lowest-index cell of
// each component is pinned to zero).
#include "dm_common.cuh"

namespace dm {

namespace {

// pivot search, row swap, pivot-row scaling and factor column of step k on the
// augmented n x 2n matrix W (one block)
__global__ void k_gj_pivot(double* __restrict__ W, int n, int k, double* __restrict__ fac, int* __restrict__ flag) {
    __shared__ double best[1024];
    __shared__ int bidx[1024];
    const int t = threadIdx.x;
    const int n2 = 2 * n;
    double bv = -1.0;
    int bi = k;
    for (int i = k + t; i < n; i += blockDim.x) {
        const double v = fabs(W[(long long)i * n2 + k]);
        if (v > bv) { bv = v; bi = i; }
    }
    best[t] = bv;
    bidx[t] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s) {
            if (best[t + s] > best[t] || (best[t + s] == best[t] && bidx[t + s] < bidx[t])) {
                best[t] = best[t + s];
                bidx[t] = bidx[t + s];
            }
        }
        __syncthreads();
    }
    const int piv = bidx[0];
    if (!(best[0] > 1e-300)) {
        if (t == 0) *flag = 1;
        return;
    }
    if (piv != k) {
        for (int j = t; j < n2; j += blockDim.x) {
            const double a = W[(long long)k * n2 + j];
            W[(long long)k * n2 + j] = W[(long long)piv * n2 + j];
            W[(long long)piv * n2 + j] = a;
        }
    }
    __syncthreads();
    const double inv = 1.0 / W[(long long)k * n2 + k];
    __syncthreads();
    for (int j = t; j < n2; j += blockDim.x) W[(long long)k * n2 + j] *= inv;
    __syncthreads();
    for (int i = t; i < n; i += blockDim.x) fac[i] = (i == k) ? 0.0 : W[(long long)i * n2 + k];
}

__global__ void k_gj_eliminate(double* __restrict__ W, int n, int k, const double* __restrict__ fac,
                               const int* __restrict__ flag) {
    if (*flag) return;
    const int n2 = 2 * n;
    const int i = blockIdx.y;
    const double f = fac[i];
    if (f == 0.0) return;
    for (int j = k + blockIdx.x * blockDim.x + threadIdx.x; j < n2; j += gridDim.x * blockDim.x)
        W[(long long)i * n2 + j] -= f * W[(long long)k * n2 + j];
}

__global__ void k_gj_init(const double* __restrict__ M, double* __restrict__ W, int n) {
    const long long tot = 2ll * n * n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / (2 * n)), j = (int)(t % (2 * n));
        W[t] = j < n ? M[(long long)i * n + j] : (j - n == i ? 1.0 : 0.0);
    }
}
__global__ void k_gj_extract(const double* __restrict__ W, double* __restrict__ M, int n) {
    const long long tot = (long long)n * n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        M[t] = W[(long long)i * 2 * n + n + j];
    }
}

template <typename T>
__global__ void k_gather(int n, const int* __restrict__ list, const unsigned char* __restrict__ zero_rows,
                         const T* __restrict__ f, double* __restrict__ out) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        out[r] = (zero_rows && zero_rows[r]) ? 0.0 : (double)to_c(f[list[r]]);
}

// out = M in  (one warp per row; FP64 or FP32 matrix, FP64 accumulation)
__global__ void k_dense_mv(int n, const double* __restrict__ M64, const float* __restrict__ M32,
                           const double* __restrict__ in, double* __restrict__ out) {
    const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double s = 0.0;
    if (M64) {
        for (int c = lane; c < n; c += 32) s += M64[(long long)row * n + c] * in[c];
    } else {
        for (int c = lane; c < n; c += 32) s += (double)M32[(long long)row * n + c] * in[c];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[row] = s;
}

template <typename T>
__global__ void k_scatter(int n, const int* __restrict__ list, const double* __restrict__ in, T* __restrict__ x) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        x[list[r]] = to_store<T>(in[r]);
}

__device__ int find_in_list(const int* list, int n, int key) {
    int lo = 0, hi = n - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int v = list[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// label propagation (single block); list sorted ascending (natural order)
__global__ void k_components(Grid3 g, const double* __restrict__ A, const int* __restrict__ list, int n,
                             int* __restrict__ label, unsigned char* __restrict__ pinned) {
    __shared__ int changed;
    for (int r = threadIdx.x; r < n; r += blockDim.x) label[r] = r;
    __syncthreads();
    const int X = 1, Y = g.sx, Z = g.sxy, N = g.np;
    for (int it = 0; it < n + 1; ++it) {
        if (threadIdx.x == 0) changed = 0;
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            const int p = list[r];
            int best = label[r];
            // neighbours across open faces: (face index, neighbour cell)
            const int faces[6] = {p, p + X, N + p, N + p + Y, 2 * N + p, 2 * N + p + Z};
            const int nbr[6] = {p - X, p + X, p - Y, p + Y, p - Z, p + Z};
            for (int f = 0; f < 6; ++f) {
                if (A[faces[f]] > 0.0) {
                    const int pos = find_in_list(list, n, nbr[f]);
                    if (pos >= 0) best = min(best, label[pos]);
                }
            }
            if (best < label[r]) {
                label[r] = best;
                changed = 1;
            }
        }
        __syncthreads();
        if (!changed) break;
        __syncthreads();
    }
    // components with an open face on the outer wall (a magnetic symmetry
    // plane) are regular: the potential beyond the wall is zero.  pinned[]
    // first marks their roots, then takes the final flags.
    for (int r = threadIdx.x; r < n; r += blockDim.x) pinned[r] = 0;
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const int p = list[r];
        const int i = (p - g.off0) % g.sx, j = ((p - g.off0) / g.sx) % g.sy, k = (p - g.off0) / g.sxy;
        const bool wall = (i == 0 && A[p] > 0.0) || (i == g.nx - 1 && A[p + X] > 0.0) ||
                          (j == 0 && A[N + p] > 0.0) || (j == g.ny - 1 && A[N + p + Y] > 0.0) ||
                          (k == 0 && A[2 * N + p] > 0.0) || (k == g.nz - 1 && A[2 * N + p + Z] > 0.0);
        if (wall) pinned[label[r]] = 2;   // benign race: every writer stores the same value
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const bool root = label[r] == r;
        pinned[r] = (root && pinned[r] != 2) ? 1 : 0;
    }
}

}  // namespace

bool dense_inverse(double* M, int n, double* work, int* d_flag, cudaStream_t s) {
    double* W = work;
    double* fac = work + 2ll * n * n;
    DM_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), s));
    launch("k_gj_init", k_gj_init, 256, 256, 0, s, M, W, n);
    const int bx = std::max(1, std::min(8, (2 * n + 255) / 256));
    for (int k = 0; k < n; ++k) {
        launch("k_gj_pivot", k_gj_pivot, 1, 1024, 0, s, W, n, k, fac, d_flag);
        launch("k_gj_eliminate", k_gj_eliminate, dim3(bx, n), 256, 0, s, W, n, k, fac, d_flag);
    }
    launch("k_gj_extract", k_gj_extract, 256, 256, 0, s, W, M, n);
    int h = 0;
    DM_CUDA(cudaMemcpyAsync(&h, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    return h == 0;
}

template <typename T>
void dense_coarse_solve(const double* Minv64, const float* Minv32, int n, const int* list, const unsigned char* zero_rows,
                        const T* f, T* x, double* tmp_in, double* tmp_out, cudaStream_t s) {
    if (n <= 0) return;
    const int b = (n + 255) / 256;
    launch("k_gather", k_gather<T>, b, 256, 0, s, n, list, zero_rows, f, tmp_in);
    launch("k_dense_mv", k_dense_mv, (n + 7) / 8, 256, 0, s, n, Minv64, Minv32, tmp_in, tmp_out);
    launch("k_scatter", k_scatter<T>, b, 256, 0, s, n, list, tmp_out, x);
}

void cell_components_pin(const Grid3& g, const double* A, const int* list, int n, int* label, unsigned char* pinned,
                         cudaStream_t s) {
    if (n <= 0) return;
    launch("k_components", k_components, 1, 512, 0, s, g, A, list, n, label, pinned);
}

template void dense_coarse_solve<double>(const double*, const float*, int, const int*, const unsigned char*,
                                         const double*, double*, double*, double*, cudaStream_t);
template void dense_coarse_solve<float>(const double*, const float*, int, const int*, const unsigned char*,
                                        const float*, float*, double*, double*, cudaStream_t);
template void dense_coarse_solve<__nv_bfloat16>(const double*, const float*, int, const int*, const unsigned char*,
                                                const __nv_bfloat16*, __nv_bfloat16*, double*, double*, cudaStream_t);

}  // namespace dm
