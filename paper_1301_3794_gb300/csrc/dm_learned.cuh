// Learned smoother network state (see dm_learned.cu for the definition).
#pragma once

#include "dm_common.cuh"

namespace dm {

struct LearnedNet {
    static constexpr int CIN_ = 8, HID = 16, COUT_ = 3;
    static constexpr int kDwBlocks = 304;           // 2 x 152 SMs: blocks of the weight-gradient reduction
    Grid3 g{};
    DBuf<float> W, G, M1, M2;                       // parameters [W1 | W2 | W3], gradient, Adam moments
    DBuf<__nv_bfloat16> X, H1, H2, dY, dH1, dH2;    // activations and their gradients, [np][C]
    DBuf<float> Y, E, loss_part, dw_part;           // output, target, reduction scratch
    int step = 0;

    static constexpr size_t n1() { return 27ull * CIN_ * HID; }
    static constexpr size_t n2() { return 27ull * HID * HID; }
    static constexpr size_t n3() { return 27ull * HID * COUT_; }
    static constexpr size_t n_params() { return n1() + n2() + n3(); }
    static constexpr size_t off2() { return n1(); }
    static constexpr size_t off3() { return n1() + n2(); }
    float* w1() { return W.get(); }
    float* w2() { return W.get() + off2(); }
    float* w3() { return W.get() + off3(); }

    void init_params();
    void alloc(const Grid3& grid);                 // activation buffers for a node grid
    // X from a residual r (padded face vector in precision r_prec: 0 f64, 1 f32, 2 bf16) scaled by inv_scale
    void features(const double* A, const double* V, double inv_scale, const void* r, int r_prec, cudaStream_t s);
    void forward(cudaStream_t s);
    float loss(const double* A, double msum, cudaStream_t s);   // needs E; writes dY
    void backward(cudaStream_t s);                               // G = dloss/dW
    void adam(float lr, cudaStream_t s);
    template <typename T>
    void add_correction(const double* A, double scale, T* z, cudaStream_t s);
    void set_X(const float* nat_dev, cudaStream_t s);       // features from a natural [nodes][8] device array
    void set_E(const float* nat_dev, cudaStream_t s);       // targets from a natural [nodes][3] device array
    void target_from(const float* e_pad, const double* A, double inv, cudaStream_t s);
    // Residual objective on the fine level: with y = h2 Y on the open faces and
    // r the (padded, FP32) residual, loss = 0.5 |r inv_scale - K y|^2 / msum over
    // the open faces (K = o's operator, FP32); writes dY = dloss/dY.  ybuf, kbuf:
    // padded FP32 face scratch.
    float residual_loss(const VecOp<float, float>& o, const double* A, const float* r, double inv_scale, double h2,
                        float* ybuf, float* kbuf, double msum, cudaStream_t s);
};

// sum of squares of a padded vector of n entries (host result)
template <typename T>
double sumsq(long long n, const T* x, cudaStream_t s);
// (x . y, y . y) over n entries: nb block partials in part_dev / part_host
// (pinned), summed on the host in a fixed order
template <typename T>
void dot2(long long n, const T* x, const T* y, double* part_dev, double* part_host, int nb, double out[2],
          cudaStream_t s);
// z += a c over n entries
template <typename T>
void axpy_store(long long n, double a, const T* c, T* z, cudaStream_t s);

}  // namespace dm
