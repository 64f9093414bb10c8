// Learned smoother network state (see dm_learned.cu for the definition).
#pragma once

#include "dm_common.cuh"

namespace dm {

// Channel-blocked activation layout: channel c of node p (padded node index)
// at element ((c / 8) npe + marg + p) * 8 + c % 8 (BF16).  Each block of eight
// channels is preceded and followed by marg zero nodes, so a 3x3x3 window
// around any 128-node tile lies inside the buffer.
struct ActLayout {
    int np = 0, marg = 0, npe = 0;
    __host__ __device__ size_t at(int cb, int p) const { return ((size_t)cb * npe + marg + p) * 8; }
    size_t elems(int cb) const { return (size_t)cb * npe * 8; }
};
ActLayout act_layout(const Grid3& g);

// Tensor-core convolution (dm_conv_tc.cu).  Weight tiles: BF16, two 16 x 16
// tiles per MMA step (the weight's BF16 rounding and the BF16 rounding of the
// rest; 512 values a step, conv_wtile_steps(cb) steps), made by conv_pack_weights
// from FP32 weights W[27][wcin][wcout] (flip = 1: the adjoint conv, whose
// input has cin = wcout channels and output cout = wcin channels).
int conv_wtile_steps(int cb);
void conv_pack_weights(const float* W, int wcin, int wcout, int cin, int cout, int cb, int flip, __nv_bfloat16* out,
                       cudaStream_t s);
// epi 0: out = relu(conv) (BF16, 16 channels); 1: out = conv * (mask > 0)
// (BF16, 16 channels); 2: outY[p][0..2] = conv (FP32).  cb: input channel
// blocks (1: up to 8 channels, 2: 16).  err: device flag set when a wait of
// the kernel timed out (0 = fine).
void conv_tc(const Grid3& g, const ActLayout& L, int cb, int epi, const __nv_bfloat16* in, const __nv_bfloat16* wt,
             const __nv_bfloat16* mask, __nv_bfloat16* out, float* outY, int* err, cudaStream_t s);
// weight gradient dW[t][ci][co] = sum_p in[p + d_t, ci] dy[p, co] on tensor
// cores: cb_in input channel blocks (cin channels), dy with cout <= 16
// channels in cb_out blocks; part: per-CTA partials (conv_dw_tc_parts() x
// 27 x 16 x 16 floats), summed in CTA order into dW ([27][cin][cout]).
int conv_dw_tc_parts();
void conv_dw_tc(const Grid3& g, const ActLayout& L, int cb_in, int cin, const __nv_bfloat16* in, int cb_out, int cout,
                const __nv_bfloat16* dy, float* part, float* dW, int* err, cudaStream_t s);

struct LearnedNet {
    static constexpr int CIN_ = 8, HID = 16, COUT_ = 3;
    Grid3 g{};
    ActLayout L{};
    DBuf<float> W, G, M1, M2;                       // parameters [W1 | W2 | W3], gradient, Adam moments
    DBuf<__nv_bfloat16> X, H1, H2, dY, dH1, dH2;    // activations and their gradients (ActLayout)
    DBuf<__nv_bfloat16> wt1, wt2, wt3, wt3a, wt2a;  // weight tiles: forward layers, adjoints of layers 3, 2
    DBuf<float> Y, E, loss_part, dw_part;           // output [np][3], target [np][3], reduction scratch
    DBuf<int> err;                                  // conv kernels' timeout flag
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
    void check(cudaStream_t s);                                  // throws if a conv kernel timed out
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
