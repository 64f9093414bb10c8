// Learned smoother: a 3-layer 3x3x3 convolutional network on the node grid of
// the fine level (a design of this library; the paper has no learned part).
//
//   H1 = relu(conv(X, W1)),  H2 = relu(conv(H1, W2)),  Y = conv(H2, W3)
//
// conv is a zero-padded 3x3x3 cross-correlation without bias:
//   conv(X, W)[p, o] = sum_{a,b,c} sum_q W[a,b,c,q,o] X[p + (c-1, b-1, a-1), q]
// (a along k, b along j, c along i).  X has 8 channels: the residual on the
// node's x, y, z faces divided by its RMS, the face fractions A_x, A_y, A_z,
// the cell fraction V, and a zero channel.  Y has 3 channels: the predicted
// error on the node's faces in units of RMS(r) * h^2.
//
// Activations are BF16 in the channel-blocked layout of ActLayout on the
// padded node grid (the ghost layer and the margins give the zero padding);
// weights, accumulation, losses and the optimiser state are FP32, and the
// tensor cores multiply BF16 copies of the weights.  The convolutions, their
// adjoints and the weight gradients are implicit GEMMs on the tensor cores
// (dm_conv_tc.cu); the weight gradient is reduced in a fixed order (per-CTA
// partials, then a sum in CTA order), so training is deterministic.
#include "dm_common.cuh"

#include "dm_learned.cuh"

#include <atomic>
#include <cmath>

namespace dm {

namespace {

constexpr int LX = TX, LY = TY, LZ = TZ;                 // node tile of the elementwise kernels

// column sums of part[nb][n] in block order
__global__ void k_colsum(const float* __restrict__ part, int nb, int n, float* __restrict__ out) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n) return;
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part[(size_t)b * n + w];
    out[w] = s;
}

// input features of every node: residual / scale on the three faces, A_x, A_y, A_z, V, 0
template <typename T>
__global__ void k_features(Grid3 g, ActLayout L, const T* __restrict__ r, const double* __restrict__ A,
                           const double* __restrict__ V, double inv_scale, __nv_bfloat16* __restrict__ X) {
    const int i = blockIdx.x * LX + threadIdx.x, j = blockIdx.y * LY + threadIdx.y, k = blockIdx.z * LZ + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int p = g.idx(i, j, k);
    __align__(16) __nv_bfloat16 x[8];
    for (int c = 0; c < 3; ++c) {
        const double a = A[c * g.np + p];
        x[c] = __float2bfloat16(a > 0.0 ? (float)(to_c(r[c * g.np + p]) * inv_scale) : 0.f);
        x[3 + c] = __float2bfloat16((float)a);
    }
    x[6] = __float2bfloat16((float)V[p]);
    x[7] = __float2bfloat16(0.f);
    *reinterpret_cast<uint4*>(X + L.at(0, p)) = *reinterpret_cast<const uint4*>(x);
}

// z += scale * Y on the open faces (Y: [np][3] fp32)
template <typename T>
__global__ void k_add_correction(Grid3 g, const float* __restrict__ Y, const double* __restrict__ A, double scale,
                                 T* __restrict__ z) {
    const int i = blockIdx.x * LX + threadIdx.x, j = blockIdx.y * LY + threadIdx.y, k = blockIdx.z * LZ + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int p = g.idx(i, j, k);
    for (int c = 0; c < 3; ++c) {
        const int q = c * g.np + p;
        if (A[q] > 0.0) z[q] = to_store<T>((double)to_c(z[q]) + scale * (double)Y[(size_t)p * 3 + c]);
    }
}

// loss = 0.5 sum M (Y - E)^2 / sum M (block partials) and dY = M (Y - E) / sum M (bf16)
__global__ void k_mse(Grid3 g, ActLayout L, const float* __restrict__ Y, const float* __restrict__ E,
                      const double* __restrict__ A, float inv_msum, __nv_bfloat16* __restrict__ dY,
                      float* __restrict__ part) {
    __shared__ float red[256];
    const int i = blockIdx.x * LX + threadIdx.x, j = blockIdx.y * LY + threadIdx.y, k = blockIdx.z * LZ + threadIdx.z;
    const int tid = threadIdx.x + LX * (threadIdx.y + LY * threadIdx.z);
    float l = 0.f;
    if (i <= g.nx && j <= g.ny && k <= g.nz) {
        const int p = g.idx(i, j, k);
        for (int c = 0; c < 3; ++c) {
            const float m = A[c * g.np + p] > 0.0 ? 1.f : 0.f;
            const float d = m * (Y[(size_t)p * 3 + c] - E[(size_t)p * 3 + c]);
            l += 0.5f * d * d;
            dY[L.at(0, p) + c] = __float2bfloat16(d * inv_msum);
        }
    }
    red[tid] = l;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (tid < s) red[tid] += red[tid + s];
        __syncthreads();
    }
    if (tid == 0) part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = red[0] * inv_msum;
}

// res = mask (r inv - Ky) in place of Ky, and block partials of 0.5 |res|^2 / msum
__global__ void k_res_loss(long long n, const float* __restrict__ r, float inv, const double* __restrict__ A,
                           float* __restrict__ ky, float inv_msum, float* __restrict__ part) {
    __shared__ float red[256];
    float l = 0.f;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const float v = A[q] > 0.0 ? r[q] * inv - ky[q] : 0.f;
        ky[q] = v;
        l += 0.5f * v * v;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0] * inv_msum;
}
// dY = a g on the open faces of each node (gathered to node-channel order)
__global__ void k_grad_gather(Grid3 g, ActLayout L, const float* __restrict__ gv, const double* __restrict__ A,
                              float a, __nv_bfloat16* __restrict__ dY) {
    const int i = blockIdx.x * LX + threadIdx.x, j = blockIdx.y * LY + threadIdx.y, k = blockIdx.z * LZ + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int p = g.idx(i, j, k);
    for (int c = 0; c < 3; ++c) {
        const int q = c * g.np + p;
        dY[L.at(0, p) + c] = __float2bfloat16(A[q] > 0.0 ? a * gv[q] : 0.f);
    }
}

__global__ void k_adam(int n, float* __restrict__ w, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gr = grad[t];
    const float mt = b1 * m[t] + (1.f - b1) * gr;
    const float vt = b2 * v[t] + (1.f - b2) * gr * gr;
    m[t] = mt;
    v[t] = vt;
    w[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

// natural node array (i fastest, channel last) -> X in the blocked layout (8 channels)
__global__ void k_pack_X(Grid3 g, ActLayout L, const float* __restrict__ nat, __nv_bfloat16* __restrict__ X) {
    const int i = blockIdx.x * LX + threadIdx.x, j = blockIdx.y * LY + threadIdx.y, k = blockIdx.z * LZ + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const long long n = i + (long long)(g.nx + 1) * (j + (long long)(g.ny + 1) * k);
    const int p = g.idx(i, j, k);
    for (int c = 0; c < 8; ++c) X[L.at(0, p) + c] = __float2bfloat16(nat[n * 8 + c]);
}
// natural node array -> [np][C] FP32 on the padded grid
__global__ void k_pack_nodes_f32(Grid3 g, int C, const float* __restrict__ nat, float* __restrict__ pad) {
    const int i = blockIdx.x * LX + threadIdx.x, j = blockIdx.y * LY + threadIdx.y, k = blockIdx.z * LZ + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const long long n = i + (long long)(g.nx + 1) * (j + (long long)(g.ny + 1) * k);
    const int p = g.idx(i, j, k);
    for (int c = 0; c < C; ++c) pad[(size_t)p * C + c] = nat[n * C + c];
}

// training target: E[p][c] = e_c[p] * inv on open faces (e: padded fp32 face vector)
__global__ void k_target(Grid3 g, const float* __restrict__ e, const double* __restrict__ A, double inv,
                         float* __restrict__ E) {
    const int i = blockIdx.x * LX + threadIdx.x, j = blockIdx.y * LY + threadIdx.y, k = blockIdx.z * LZ + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int p = g.idx(i, j, k);
    for (int c = 0; c < 3; ++c) {
        const int q = c * g.np + p;
        E[(size_t)p * 3 + c] = A[q] > 0.0 ? (float)(e[q] * inv) : 0.f;
    }
}

// block partials of sum x^2 over a padded face vector of any storage type
template <typename T>
__global__ void k_sumsq(long long n, const T* __restrict__ x, double* __restrict__ part) {
    __shared__ double red[256];
    double a = 0.0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        const double v = (double)to_c(x[r]);
        a += v * v;
    }
    red[threadIdx.x] = a;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void k_sum_d(const double* __restrict__ part, int n, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s += part[b];
        *out = s;
    }
}

inline dim3 node_blocks(const Grid3& g) {
    return dim3((g.nx + LX) / LX, (g.ny + LY) / LY, (g.nz + LZ) / LZ);
}

}  // namespace

// ---------------------------------------------------------------------------

void LearnedNet::alloc(const Grid3& grid) {
    if (g.np == grid.np && g.nx == grid.nx && g.ny == grid.ny && g.nz == grid.nz && X.get()) return;
    g = grid;
    L = act_layout(g);
    const size_t np = (size_t)g.np;
    X.alloc(L.elems(1));
    H1.alloc(L.elems(2));
    H2.alloc(L.elems(2));
    dY.alloc(L.elems(1));
    dH1.alloc(L.elems(2));
    dH2.alloc(L.elems(2));
    Y.alloc(np * COUT_);
    E.alloc(np * COUT_);
    wt1.alloc((size_t)conv_wtile_steps(1) * 512);
    wt2.alloc((size_t)conv_wtile_steps(2) * 512);
    wt3.alloc((size_t)conv_wtile_steps(2) * 512);
    wt3a.alloc((size_t)conv_wtile_steps(1) * 512);
    wt2a.alloc((size_t)conv_wtile_steps(2) * 512);
    err.alloc(1);
    const dim3 nb = node_blocks(g);
    loss_part.alloc((size_t)nb.x * nb.y * nb.z);
    dw_part.alloc((size_t)conv_dw_tc_parts() * 27 * 256);
}

void LearnedNet::init_params() {
    W.alloc(n_params());
    G.alloc(n_params());
    M1.alloc(n_params());
    M2.alloc(n_params());
}

void LearnedNet::features(const double* A, const double* V, double inv_scale, const void* r, int r_prec,
                          cudaStream_t s) {
    const dim3 nb = node_blocks(g);
    const dim3 bl(LX, LY, LZ);
    if (r_prec == 0)
        launch("learned_features", k_features<double>, nb, bl, 0, s, g, L, (const double*)r, A, V, inv_scale, X.get());
    else if (r_prec == 1)
        launch("learned_features", k_features<float>, nb, bl, 0, s, g, L, (const float*)r, A, V, inv_scale, X.get());
    else
        launch("learned_features", k_features<__nv_bfloat16>, nb, bl, 0, s, g, L, (const __nv_bfloat16*)r, A, V,
               inv_scale, X.get());
}

// conv_tc epilogues
constexpr int kEpiRelu = 0, kEpiMask = 1, kEpiOut = 2;

void LearnedNet::forward(cudaStream_t s) {
    conv_pack_weights(w1(), CIN_, HID, CIN_, HID, 1, 0, wt1.get(), s);
    conv_pack_weights(w2(), HID, HID, HID, HID, 2, 0, wt2.get(), s);
    conv_pack_weights(w3(), HID, COUT_, HID, COUT_, 2, 0, wt3.get(), s);
    conv_tc(g, L, 1, kEpiRelu, X.get(), wt1.get(), nullptr, H1.get(), nullptr, err.get(), s);
    conv_tc(g, L, 2, kEpiRelu, H1.get(), wt2.get(), nullptr, H2.get(), nullptr, err.get(), s);
    conv_tc(g, L, 2, kEpiOut, H2.get(), wt3.get(), nullptr, nullptr, Y.get(), err.get(), s);
}

void LearnedNet::backward(cudaStream_t s) {
    // dW3 = dW(H2, dY); dH2 = conv^T(dY, W3) * (H2 > 0); dW2 = dW(H1, dH2); dH1 = conv^T(dH2, W2) * (H1 > 0);
    // dW1 = dW(X, dH1)
    conv_pack_weights(w3(), HID, COUT_, COUT_, HID, 1, 1, wt3a.get(), s);
    conv_pack_weights(w2(), HID, HID, HID, HID, 2, 1, wt2a.get(), s);
    conv_dw_tc(g, L, 2, HID, H2.get(), 1, COUT_, dY.get(), dw_part.get(), G.get() + off3(), err.get(), s);
    conv_tc(g, L, 1, kEpiMask, dY.get(), wt3a.get(), H2.get(), dH2.get(), nullptr, err.get(), s);
    conv_dw_tc(g, L, 2, HID, H1.get(), 2, HID, dH2.get(), dw_part.get(), G.get() + off2(), err.get(), s);
    conv_tc(g, L, 2, kEpiMask, dH2.get(), wt2a.get(), H1.get(), dH1.get(), nullptr, err.get(), s);
    conv_dw_tc(g, L, 1, CIN_, X.get(), 2, HID, dH1.get(), dw_part.get(), G.get(), err.get(), s);
}

void LearnedNet::check(cudaStream_t s) {
    int h = 0;
    DM_CUDA(cudaMemcpyAsync(&h, err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    if (h != 0) {
        DM_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
        throw Error(DM_ERR_TIMEOUT, "learned network: a tensor-core conv kernel timed out waiting (code " +
                                        std::to_string(h) + ")");
    }
}

float LearnedNet::loss(const double* A, double msum, cudaStream_t s) {
    const dim3 nb = node_blocks(g);
    launch("learned_mse", k_mse, nb, dim3(LX, LY, LZ), 0, s, g, L, Y.get(), E.get(), A,
           (float)(1.0 / std::max(msum, 1.0)), dY.get(), loss_part.get());
    const int n = nb.x * nb.y * nb.z;
    DBuf<float> tot(1);
    launch("learned_mse_sum", k_colsum, 1, 256, 0, s, loss_part.get(), n, 1, tot.get());
    float h = 0.f;
    DM_CUDA(cudaMemcpyAsync(&h, tot.get(), sizeof(float), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    return h;
}

float LearnedNet::residual_loss(const VecOp<float, float>& o, const double* A, const float* r, double inv_scale,
                                double h2, float* ybuf, float* kbuf, double msum, cudaStream_t s) {
    const long long n = 3ll * g.np;
    // y = h^2 Y on the open faces, K y
    DM_CUDA(cudaMemsetAsync(ybuf, 0, sizeof(float) * (size_t)n, s));
    add_correction<float>(A, h2, ybuf, s);
    vec_stencil<float, float>(o, ST_APPLY, ybuf, nullptr, kbuf, 0.0, s);
    // res = r / RMS(r) - K y and the loss
    const int nb = 152 * 4;
    if (loss_part.n < (size_t)nb) loss_part.alloc(nb);
    const float inv_m = (float)(1.0 / std::max(msum, 1.0));
    launch("learned_res_loss", k_res_loss, nb, 256, 0, s, n, r, (float)inv_scale, A, kbuf, inv_m, loss_part.get());
    DBuf<float> tot(1);
    launch("learned_mse_sum", k_colsum, 1, 256, 0, s, loss_part.get(), nb, 1, tot.get());
    // dloss/dy = -K res / msum (K symmetric), dloss/dY = h^2 dloss/dy
    vec_stencil<float, float>(o, ST_APPLY, kbuf, nullptr, ybuf, 0.0, s);
    launch("learned_grad_gather", k_grad_gather, node_blocks(g), dim3(LX, LY, LZ), 0, s, g, L, ybuf, A,
           (float)(-h2 * inv_m), dY.get());
    float h = 0.f;
    DM_CUDA(cudaMemcpyAsync(&h, tot.get(), sizeof(float), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    return h;
}

void LearnedNet::adam(float lr, cudaStream_t s) {
    ++step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)step), c2 = 1.f - std::pow(b2, (float)step);
    const int n = (int)n_params();
    launch("learned_adam", k_adam, (n + 255) / 256, 256, 0, s, n, W.get(), G.get(), M1.get(), M2.get(), lr, b1, b2,
           1e-8f, c1, c2);
}

void LearnedNet::set_X(const float* nat_dev, cudaStream_t s) {
    launch("learned_pack", k_pack_X, node_blocks(g), dim3(LX, LY, LZ), 0, s, g, L, nat_dev, X.get());
}
void LearnedNet::set_E(const float* nat_dev, cudaStream_t s) {
    launch("learned_pack", k_pack_nodes_f32, node_blocks(g), dim3(LX, LY, LZ), 0, s, g, COUT_, nat_dev, E.get());
}
void LearnedNet::target_from(const float* e_pad, const double* A, double inv, cudaStream_t s) {
    launch("learned_target", k_target, node_blocks(g), dim3(LX, LY, LZ), 0, s, g, e_pad, A, inv, E.get());
}

template <typename T>
double sumsq(long long n, const T* x, cudaStream_t s) {
    const int nb = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 4));
    DBuf<double> part(nb), out(1);
    launch("learned_sumsq", k_sumsq<T>, nb, 256, 0, s, n, x, part.get());
    launch("learned_sumsq", k_sum_d, 1, 32, 0, s, part.get(), nb, out.get());
    double h = 0.0;
    DM_CUDA(cudaMemcpyAsync(&h, out.get(), sizeof(double), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    return h;
}
template double sumsq<double>(long long, const double*, cudaStream_t);
template double sumsq<float>(long long, const float*, cudaStream_t);
template double sumsq<__nv_bfloat16>(long long, const __nv_bfloat16*, cudaStream_t);

// block partials of (x . y, y . y) over n entries of two vectors of storage type T
template <typename T>
__global__ void k_dot2(long long n, const T* __restrict__ x, const T* __restrict__ y, double* __restrict__ part) {
    __shared__ double ra[256], rb[256];
    double a = 0.0, b = 0.0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        const double xv = (double)to_c(x[r]), yv = (double)to_c(y[r]);
        a += xv * yv;
        b += yv * yv;
    }
    ra[threadIdx.x] = a;
    rb[threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            ra[threadIdx.x] += ra[threadIdx.x + s];
            rb[threadIdx.x] += rb[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = ra[0];
        part[2 * blockIdx.x + 1] = rb[0];
    }
}
// z += a c over n entries
template <typename T>
__global__ void k_axpy_store(long long n, double a, const T* __restrict__ c, T* __restrict__ z) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        z[r] = to_store<T>((double)to_c(z[r]) + a * (double)to_c(c[r]));
}

template <typename T>
void dot2(long long n, const T* x, const T* y, double* part_dev, double* part_host, int nb, double out[2],
          cudaStream_t s) {
    launch("learned_dot2", k_dot2<T>, nb, 256, 0, s, n, x, y, part_dev);
    DM_CUDA(cudaMemcpyAsync(part_host, part_dev, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    out[0] = out[1] = 0.0;
    for (int b = 0; b < nb; ++b) {
        out[0] += part_host[2 * b];
        out[1] += part_host[2 * b + 1];
    }
}
template <typename T>
void axpy_store(long long n, double a, const T* c, T* z, cudaStream_t s) {
    const int nb = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8));
    launch("learned_axpy", k_axpy_store<T>, nb, 256, 0, s, n, a, c, z);
}
#define DM_INST(T)                                                                                              \
    template void dot2<T>(long long, const T*, const T*, double*, double*, int, double[2], cudaStream_t);       \
    template void axpy_store<T>(long long, double, const T*, T*, cudaStream_t);
DM_INST(double)
DM_INST(float)
DM_INST(__nv_bfloat16)
#undef DM_INST

template <typename T>
void LearnedNet::add_correction(const double* A, double scale, T* z, cudaStream_t s) {
    launch("learned_correct", k_add_correction<T>, node_blocks(g), dim3(LX, LY, LZ), 0, s, g, Y.get(), A, scale, z);
}
template void LearnedNet::add_correction<double>(const double*, double, double*, cudaStream_t);
template void LearnedNet::add_correction<float>(const double*, double, float*, cudaStream_t);
template void LearnedNet::add_correction<__nv_bfloat16>(const double*, double, __nv_bfloat16*, cudaStream_t);

}  // namespace dm
