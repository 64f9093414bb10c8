// Vector kernels of the Krylov solvers: (weighted) multi-dot products with a
// deterministic two-pass reduction, multi-AXPY, basis recombination, copies,
// precision conversion and a counter-based random fill.
//
// The weighted dot sum_r w_r u_r v_r with w = A (the face fractions) is the
// inner product of Eq. bInner in which P_DM (Eq. proj) is an orthogonal
// projection and the shift-inverted operator of Eq. fullMat is self-adjoint.
//
// Every kernel runs over a Domain: either the list of active 32 x 4 x 2 node
// tiles of a level (entries outside them are zero in every vector and are
// neither read nor written), or, with no tile list, the whole array.
#include "dm_common.cuh"

namespace dm {

namespace {

constexpr int kThreads = 256;      // = TX * TY * TZ: one tile per block pass
constexpr int kChunk = 8;          // columns per pass of the multi-dot
constexpr int kMaxBlocks = 152 * 4;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// partial[b * ldp + c0 + c] = sum over this block's entries of w * V_c * x
__global__ void k_mdot_partial(Domain d, int m, const double* __restrict__ V, long long ld,
                               const double* __restrict__ x, const double* __restrict__ w, double* __restrict__ partial,
                               int ldp, int self) {
    __shared__ double red[kThreads / 32][kChunk];
    __shared__ double red_self[kThreads / 32];
    double acc_self = 0.0;
    for (int c0 = 0; c0 < m; c0 += kChunk) {
        const int nc = min(kChunk, m - c0);
        double acc[kChunk];
#pragma unroll
        for (int c = 0; c < kChunk; ++c) acc[c] = 0.0;
        const bool first = c0 == 0 && self;
        for_each_entry(d, [&](long long r) {
            const double x0 = x[r];
            const double xr = w ? x0 * w[r] : x0;
            if (first) acc_self += xr * x0;
#pragma unroll
            for (int c = 0; c < kChunk; ++c)
                if (c < nc) acc[c] += V[(c0 + c) * ld + r] * xr;
        });
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int c = 0; c < kChunk; ++c) {
            const double s = warp_sum(acc[c]);
            if (lane == 0) red[wid][c] = s;
        }
        __syncthreads();
        if (threadIdx.x < nc) {
            double s = 0.0;
            for (int k = 0; k < kThreads / 32; ++k) s += red[k][threadIdx.x];
            partial[(long long)blockIdx.x * ldp + c0 + threadIdx.x] = s;
        }
        __syncthreads();
    }
    if (self) {
        const double v = warp_sum(acc_self);
        if ((threadIdx.x & 31) == 0) red_self[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < kThreads / 32; ++k) t += red_self[k];
            partial[(long long)blockIdx.x * ldp + m] = t;
        }
    }
}

// x -= sum_c h[c] V_c (h on the device) and the block partial of sum w x^2 of the result
__global__ void k_maxpy_norm(Domain d, int m, const double* __restrict__ V, long long ld,
                             const double* __restrict__ h, double* __restrict__ x, const double* __restrict__ w,
                             double* __restrict__ partial) {
    __shared__ double hs[128];
    __shared__ double red[kThreads / 32];
    for (int c = threadIdx.x; c < m; c += blockDim.x) hs[c] = h[c];
    __syncthreads();
    double acc_self = 0.0;
    for_each_entry(d, [&](long long r) {
        double acc = 0.0;
        for (int c = 0; c < m; ++c) acc += hs[c] * V[c * ld + r];
        const double v = x[r] - acc;
        x[r] = v;
        acc_self += (w ? w[r] * v : v) * v;
    });
    const double v = warp_sum(acc_self);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) t += red[k];
        partial[blockIdx.x] = t;
    }
}

// result[c] = sum_b partial[b * ldp + c]  (one warp per column, fixed order)
__global__ void k_mdot_final(int nb, int m, const double* __restrict__ partial, int ldp, double* __restrict__ result) {
    const int c = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= m) return;
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += partial[(long long)b * ldp + c];
    s = warp_sum(s);
    if (lane == 0) result[c] = s;
}

__global__ void k_maxpy(Domain d, int m, const double* __restrict__ V, long long ld, const double* __restrict__ h,
                        double* __restrict__ x) {
    __shared__ double hs[128];
    for (int c = threadIdx.x; c < m; c += blockDim.x) hs[c] = h[c];
    __syncthreads();
    for_each_entry(d, [&](long long r) {
        double acc = 0.0;
        for (int c = 0; c < m; ++c) acc += hs[c] * V[c * ld + r];
        x[r] -= acc;
    });
}

__global__ void k_vgemm(Domain d, int m, int p, const double* __restrict__ V, long long ld,
                        const double* __restrict__ Y, int ldy, double* __restrict__ out, long long ldo) {
    extern __shared__ double Ys[];
    for (int t = threadIdx.x; t < m * p; t += blockDim.x) {
        const int c = t % m, j = t / m;
        Ys[t] = Y[c + (long long)ldy * j];
    }
    __syncthreads();
    for_each_entry(d, [&](long long r) {
        for (int j0 = 0; j0 < p; j0 += 8) {
            double acc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = 0.0;
            for (int c = 0; c < m; ++c) {
                const double v = V[c * ld + r];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j0 + j < p) acc[j] += v * Ys[c + m * (j0 + j)];
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j0 + j < p) out[(j0 + j) * ldo + r] = acc[j];
        }
    });
}

__global__ void k_axpby(Domain d, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
    for_each_entry(d, [&](long long r) { y[r] = a * x[r] + b * y[r]; });
}
__global__ void k_scale_copy(Domain d, double a, const double* __restrict__ x, double* __restrict__ y) {
    for_each_entry(d, [&](long long r) { y[r] = a * x[r]; });
}
__global__ void k_scale_inplace(Domain d, double a, double* __restrict__ y) {
    for_each_entry(d, [&](long long r) { y[r] *= a; });
}
__global__ void k_hadamard(Domain d, const double* __restrict__ a, const double* __restrict__ x,
                           double* __restrict__ y) {
    for_each_entry(d, [&](long long r) { y[r] = a[r] * x[r]; });
}
template <typename TD, typename TS>
__global__ void k_convert(Domain d, const TS* __restrict__ x, TD* __restrict__ y) {
    for_each_entry(d, [&](long long r) { y[r] = to_store<TD>(to_c(x[r])); });
}
template <typename TD>
__global__ void k_convert_coeff(long long n, const double* __restrict__ x, TD* __restrict__ y) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        y[r] = (TD)x[r];
}

// splitmix64 finaliser (Steele, Lea & Flood 2014) as a counter-based generator
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
__global__ void k_fill_random(Domain d, unsigned long long seed, const double* __restrict__ mask,
                              double* __restrict__ x) {
    for_each_entry(d, [&](long long r) {
        const unsigned long long z = mix64(seed * 0x632be59bd9b4e019ull + (unsigned long long)r);
        const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
        x[r] = (mask && !(mask[r] > 0.0)) ? 0.0 : u;
    });
}

// ---- Krylov vectors in float-float (a pair of FP32 values per entry) -------
// GB300 issues FP64 instructions at a small fraction of its FP32 rate, so
// Gram-Schmidt on FP64 vectors is bound by the FP64 pipe, not by HBM.  The
// FGMRES basis and work vector are therefore stored as hi + lo (two FP32,
// about 48 significant bits) and every dot product, update and norm on them
// runs on the FP32 pipes with error-free transforms (Dekker's product via FMA,
// Knuth's two-sum).  FP64 values enter through ff_bits, which splits a double
// with integer operations only.

// hi = the double's leading 24 significant bits (truncated), lo = the rest
// rounded to FP32; magnitudes outside the normal FP32 range give hi = 0
// (below 2^-126) or +-inf (at and above 2^128), and lo is flushed to 0 when it
// would fall below the normal FP32 range (so values under about 2^-100 keep
// only FP32 precision: callers split vectors scaled to unit norm or to the
// operator's natural scale).
__device__ __forceinline__ float2 ff_bits(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned int sgn = (unsigned int)(b >> 32) & 0x80000000u;
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    const int e = (int)(mag >> 52);                      // biased FP64 exponent
    const int fe = e - 1023 + 127;                        // biased FP32 exponent of hi
    if (fe <= 0) return make_float2(__uint_as_float(sgn), __uint_as_float(sgn));
    if (fe >= 255) return make_float2(__uint_as_float(sgn | 0x7f800000u), 0.f);
    const float hi = __uint_as_float(sgn | ((unsigned int)fe << 23) | (unsigned int)((mag >> 29) & 0x7fffffu));
    const unsigned int rem = (unsigned int)(mag & 0x1fffffffu);   // 29 low mantissa bits, weight 2^(e - 1075)
    if (rem == 0) return make_float2(hi, __uint_as_float(sgn));
    const int k = 31 - __clz(rem);                        // leading bit of rem
    const int le = k + e - 1075 + 127;                     // biased exponent of lo
    if (le <= 0) return make_float2(hi, __uint_as_float(sgn));
    unsigned int frac;
    if (k <= 23) {
        frac = (rem << (23 - k)) & 0x7fffffu;
    } else {
        // round to nearest, ties to even, on the k - 23 dropped bits
        const int sh = k - 23;
        const unsigned int keep = rem >> sh, drop = rem & ((1u << sh) - 1u), half = 1u << (sh - 1);
        unsigned int m = keep + ((drop > half || (drop == half && (keep & 1u))) ? 1u : 0u);
        if (m >> 24) return make_float2(hi, __uint_as_float(sgn | ((unsigned int)(le + 1) << 23)));
        frac = m & 0x7fffffu;
    }
    return make_float2(hi, __uint_as_float(sgn | ((unsigned int)le << 23) | frac));
}
// s + e += a * b with a = (ah, al), b = (bh, bl) (s the running sum, e the
// collected rounding errors and low-order terms)
__device__ __forceinline__ void ff_madd(float ah, float al, float bh, float bl, float& s, float& e) {
    // the _rn intrinsics are never contracted into FMAs, which would break the
    // error-free transforms
    const float p = __fmul_rn(ah, bh);
    float pe = fmaf(ah, bh, -p);
    pe = fmaf(ah, bl, pe);
    pe = fmaf(al, bh, pe);
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    e = __fadd_rn(e, __fadd_rn(err, pe));
    s = t;
}
// (hi, lo) with |lo| <= ulp(hi) / 2 from an unnormalised pair (Fast2Sum, |s| >= |e|)
__device__ __forceinline__ float2 ff_norm(float s, float e) {
    const float hi = __fadd_rn(s, e);
    return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}
__device__ __forceinline__ double ff_to_double(float2 v) { return (double)v.x + (double)v.y; }

// y = split(a x); a = 1 skips the FP64 multiply
__global__ void k_ff_split(Domain d, double a, const double* __restrict__ x, float2* __restrict__ y) {
    if (a == 1.0) for_each_entry(d, [&](long long r) { y[r] = ff_bits(x[r]); });
    else for_each_entry(d, [&](long long r) { y[r] = ff_bits(a * x[r]); });
}
// y = a x, a = (ah, al)
__global__ void k_ff_scale(Domain d, float ah, float al, const float2* __restrict__ x, float2* __restrict__ y) {
    for_each_entry(d, [&](long long r) {
        const float2 v = x[r];
        float s = 0.f, e = 0.f;
        ff_madd(ah, al, v.x, v.y, s, e);
        y[r] = ff_norm(s, e);
    });
}
template <typename T>
__global__ void k_ff_convert(Domain d, const float2* __restrict__ x, T* __restrict__ y) {
    for_each_entry(d, [&](long long r) {
        const float2 v = x[r];
        if constexpr (std::is_same<T, double>::value) y[r] = ff_to_double(v);
        else y[r] = to_store<T>(__fadd_rn(v.x, v.y));
    });
}

// partial[b * ldp + c0 + c] = sum over this block's entries of V_c x; with
// self, partial[b * ldp + m] = sum x^2
__global__ void k_ff_mdot_partial(Domain d, int m, const float2* __restrict__ V, long long ld,
                                  const float2* __restrict__ x, double* __restrict__ partial, int ldp, int self) {
    constexpr int kc = 8;
    __shared__ double red[kThreads / 32][kc];
    __shared__ double red_self[kThreads / 32];
    float ss = 0.f, se = 0.f;
    for (int c0 = 0; c0 < m; c0 += kc) {
        const int nc = min(kc, m - c0);
        float s[kc], e[kc];
#pragma unroll
        for (int c = 0; c < kc; ++c) s[c] = e[c] = 0.f;
        const bool first = c0 == 0 && self;
        for_each_entry(d, [&](long long r) {
            const float2 xs = x[r];
            if (first) ff_madd(xs.x, xs.y, xs.x, xs.y, ss, se);
#pragma unroll
            for (int c = 0; c < kc; ++c)
                if (c < nc) {
                    const float2 v = V[(c0 + c) * ld + r];
                    ff_madd(v.x, v.y, xs.x, xs.y, s[c], e[c]);
                }
        });
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int c = 0; c < kc; ++c) {
            const double t = warp_sum((double)s[c] + (double)e[c]);
            if (lane == 0) red[wid][c] = t;
        }
        __syncthreads();
        if (threadIdx.x < nc) {
            double t = 0.0;
            for (int k = 0; k < kThreads / 32; ++k) t += red[k][threadIdx.x];
            partial[(long long)blockIdx.x * ldp + c0 + threadIdx.x] = t;
        }
        __syncthreads();
    }
    if (self) {
        const double v = warp_sum((double)ss + (double)se);
        if ((threadIdx.x & 31) == 0) red_self[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < kThreads / 32; ++k) t += red_self[k];
            partial[(long long)blockIdx.x * ldp + m] = t;
        }
    }
}

// x -= sum_c h[c] V_c (h on the device, FP64) and the block partial of sum x^2
__global__ void k_ff_maxpy_norm(Domain d, int m, const float2* __restrict__ V, long long ld,
                                const double* __restrict__ h, float2* __restrict__ x, double* __restrict__ partial) {
    __shared__ float2 hs[128];
    __shared__ double red[kThreads / 32];
    for (int c = threadIdx.x; c < m; c += blockDim.x) hs[c] = ff_bits(-h[c]);
    __syncthreads();
    float ns = 0.f, ne = 0.f;
    for_each_entry(d, [&](long long r) {
        const float2 x0 = x[r];
        float s = x0.x, e = x0.y;
        for (int c = 0; c < m; ++c) {
            const float2 v = V[c * ld + r];
            ff_madd(hs[c].x, hs[c].y, v.x, v.y, s, e);
        }
        const float2 y = ff_norm(s, e);
        x[r] = y;
        ff_madd(y.x, y.y, y.x, y.y, ns, ne);
    });
    const double v = warp_sum((double)ns + (double)ne);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) t += red[k];
        partial[blockIdx.x] = t;
    }
}

inline int blocks_for(const Domain& d) {
    const long long work = d.tiles ? (long long)d.ntiles : (d.len() + kThreads - 1) / kThreads;
    return (int)std::max<long long>(1, std::min<long long>(work, kMaxBlocks));
}

}  // namespace

void reducer_init(Reducer& r, int max_cols) {
    r.cap_blocks = kMaxBlocks;
    r.max_cols = max_cols;
    DM_CUDA(cudaMalloc(&r.partial, sizeof(double) * (size_t)r.cap_blocks * max_cols));
    DM_CUDA(cudaMalloc(&r.result, sizeof(double) * (size_t)max_cols));
    DM_CUDA(cudaMallocHost(&r.host, sizeof(double) * (size_t)max_cols));
}
void reducer_free(Reducer& r) {
    if (r.partial) cudaFree(r.partial);
    if (r.result) cudaFree(r.result);
    if (r.host) cudaFreeHost(r.host);
    r = Reducer{};
}

void mdot(Reducer& red, const Domain& d, int m, const double* V, long long ld, const double* x, const double* w,
          double* host_out, cudaStream_t s) {
    DM_REQUIRE(m >= 1 && m <= red.max_cols, DM_ERR_INVALID_ARG, "mdot: too many columns");
    const int nb = blocks_for(d);
    launch("k_mdot_partial", k_mdot_partial, nb, kThreads, 0, s, d, m, V, ld, x, w, red.partial, red.max_cols, 0);
    launch("k_mdot_final", k_mdot_final, (m + 7) / 8, 256, 0, s, nb, m, red.partial, red.max_cols, red.result);
    DM_CUDA(cudaMemcpyAsync(red.host, red.result, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < m; ++c) host_out[c] = red.host[c];
}

void mdot_self(Reducer& red, const Domain& d, int m, const double* V, long long ld, const double* x, const double* w,
               double* host_out, double* self_out, cudaStream_t s) {
    DM_REQUIRE(m >= 1 && m + 1 <= red.max_cols, DM_ERR_INVALID_ARG, "mdot: too many columns");
    const int nb = blocks_for(d);
    launch("k_mdot_partial", k_mdot_partial, nb, kThreads, 0, s, d, m, V, ld, x, w, red.partial, red.max_cols, 1);
    launch("k_mdot_final", k_mdot_final, (m + 1 + 7) / 8, 256, 0, s, nb, m + 1, red.partial, red.max_cols, red.result);
    DM_CUDA(cudaMemcpyAsync(red.host, red.result, sizeof(double) * (m + 1), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < m; ++c) host_out[c] = red.host[c];
    *self_out = red.host[m];
}

double maxpy_norm(Reducer& red, const Domain& d, int m, const double* V, long long ld, double* x, const double* w,
                  cudaStream_t s) {
    DM_REQUIRE(m >= 1 && m <= 128 && m <= red.max_cols, DM_ERR_INVALID_ARG, "maxpy: too many columns");
    const int nb = blocks_for(d);
    // h = red.result (written by the preceding mdot on this stream); partials in a separate stripe
    double* part = red.partial + (size_t)red.cap_blocks * (red.max_cols - 1);
    launch("k_maxpy_norm", k_maxpy_norm, nb, kThreads, 0, s, d, m, V, ld, red.result, x, w, part);
    launch("k_mdot_final", k_mdot_final, 1, 256, 0, s, nb, 1, part, 1, red.result + red.max_cols - 1);
    DM_CUDA(cudaMemcpyAsync(red.host, red.result + red.max_cols - 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    return red.host[0];
}

void maxpy(Reducer& red, const Domain& d, int m, const double* V, long long ld, const double* h_host, double* x,
           cudaStream_t s) {
    DM_REQUIRE(m >= 1 && m <= 128 && m <= red.max_cols, DM_ERR_INVALID_ARG, "maxpy: too many columns");
    // stage h through pinned memory (the host array may be pageable)
    DM_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < m; ++c) red.host[c] = h_host[c];
    DM_CUDA(cudaMemcpyAsync(red.result, red.host, sizeof(double) * m, cudaMemcpyHostToDevice, s));
    launch("k_maxpy", k_maxpy, blocks_for(d), kThreads, 0, s, d, m, V, ld, red.result, x);
}

void ff_split(const Domain& d, double a, const double* x, float2* y, cudaStream_t s) {
    launch("k_ff_split", k_ff_split, blocks_for(d), kThreads, 0, s, d, a, x, y);
}
void ff_scale(const Domain& d, double a, const float2* x, float2* y, cudaStream_t s) {
    const float ah = (float)a;
    const float al = (float)(a - (double)ah);
    launch("k_ff_scale", k_ff_scale, blocks_for(d), kThreads, 0, s, d, ah, al, x, y);
}
template <typename T>
void ff_convert(const Domain& d, const float2* x, T* y, cudaStream_t s) {
    launch("k_ff_convert", k_ff_convert<T>, blocks_for(d), kThreads, 0, s, d, x, y);
}
template void ff_convert<double>(const Domain&, const float2*, double*, cudaStream_t);
template void ff_convert<float>(const Domain&, const float2*, float*, cudaStream_t);
template void ff_convert<__nv_bfloat16>(const Domain&, const float2*, __nv_bfloat16*, cudaStream_t);
void mdot_ff(Reducer& red, const Domain& d, int m, const float2* V, long long ld, const float2* x, double* host_out,
             double* self_out, cudaStream_t s) {
    const int self = self_out ? 1 : 0;
    DM_REQUIRE(m >= 1 && m + self <= red.max_cols, DM_ERR_INVALID_ARG, "mdot: too many columns");
    const int nb = blocks_for(d);
    launch("k_ff_mdot_partial", k_ff_mdot_partial, nb, kThreads, 0, s, d, m, V, ld, x, red.partial, red.max_cols,
           self);
    launch("k_mdot_final", k_mdot_final, (m + self + 7) / 8, 256, 0, s, nb, m + self, red.partial, red.max_cols,
           red.result);
    DM_CUDA(cudaMemcpyAsync(red.host, red.result, sizeof(double) * (m + self), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < m; ++c) host_out[c] = red.host[c];
    if (self_out) *self_out = red.host[m];
}
double maxpy_norm_ff(Reducer& red, const Domain& d, int m, const float2* V, long long ld, float2* x, cudaStream_t s) {
    DM_REQUIRE(m >= 1 && m <= 128 && m <= red.max_cols, DM_ERR_INVALID_ARG, "maxpy: too many columns");
    const int nb = blocks_for(d);
    double* part = red.partial + (size_t)red.cap_blocks * (red.max_cols - 1);
    launch("k_ff_maxpy_norm", k_ff_maxpy_norm, nb, kThreads, 0, s, d, m, V, ld, red.result, x, part);
    launch("k_mdot_final", k_mdot_final, 1, 256, 0, s, nb, 1, part, 1, red.result + red.max_cols - 1);
    DM_CUDA(cudaMemcpyAsync(red.host, red.result + red.max_cols - 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    return red.host[0];
}

void vgemm(const Domain& d, int m, int p, const double* V, long long ld, const double* Y_dev, int ldy, double* out,
           long long ldo, cudaStream_t s) {
    const size_t sm = sizeof(double) * (size_t)m * p;
    DM_REQUIRE(sm <= 48 * 1024, DM_ERR_INVALID_ARG, "vgemm: basis too large");
    launch("k_vgemm", k_vgemm, blocks_for(d), kThreads, sm, s, d, m, p, V, ld, Y_dev, ldy, out, ldo);
}

void axpby(const Domain& d, double a, const double* x, double b, double* y, cudaStream_t s) {
    launch("k_axpby", k_axpby, blocks_for(d), kThreads, 0, s, d, a, x, b, y);
}
void scale_copy(const Domain& d, double a, const double* x, double* y, cudaStream_t s) {
    if (x == y) launch("k_scale_inplace", k_scale_inplace, blocks_for(d), kThreads, 0, s, d, a, y);
    else launch("k_scale_copy", k_scale_copy, blocks_for(d), kThreads, 0, s, d, a, x, y);
}
void hadamard(const Domain& d, const double* a, const double* x, double* y, cudaStream_t s) {
    launch("k_hadamard", k_hadamard, blocks_for(d), kThreads, 0, s, d, a, x, y);
}
template <typename TD, typename TS>
void convert(const Domain& d, const TS* x, TD* y, cudaStream_t s) {
    launch("k_convert", k_convert<TD, TS>, blocks_for(d), kThreads, 0, s, d, x, y);
}
template <typename TD>
void convert_coeff(long long n, const double* x, TD* y, cudaStream_t s) {
    const int b = (int)std::max<long long>(1, std::min<long long>((n + kThreads - 1) / kThreads, kMaxBlocks));
    launch("k_convert_coeff", k_convert_coeff<TD>, b, kThreads, 0, s, n, x, y);
}
void fill_random(const Domain& d, unsigned long long seed, const double* mask, double* x, cudaStream_t s) {
    launch("k_fill_random", k_fill_random, blocks_for(d), kThreads, 0, s, d, seed, mask, x);
}
void zero(void* p, size_t bytes, cudaStream_t s) { DM_CUDA(cudaMemsetAsync(p, 0, bytes, s)); }

template void convert<float, double>(const Domain&, const double*, float*, cudaStream_t);
template void convert<double, float>(const Domain&, const float*, double*, cudaStream_t);
template void convert<__nv_bfloat16, double>(const Domain&, const double*, __nv_bfloat16*, cudaStream_t);
template void convert<double, __nv_bfloat16>(const Domain&, const __nv_bfloat16*, double*, cudaStream_t);
template void convert<double, double>(const Domain&, const double*, double*, cudaStream_t);
template void convert_coeff<float>(long long, const double*, float*, cudaStream_t);

}  // namespace dm
