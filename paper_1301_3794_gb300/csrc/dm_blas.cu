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

#include <map>
#include <mutex>

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

// partial[b] = sum over this block's share of the listed entries of x[q] y[q]
// (times w[q] if w is given): a flat loop over an ascending index list, every
// load independent of the previous one (the tile loop of k_mdot_partial waits
// for each tile's index)
__global__ void k_dot_list(long long n, const int* __restrict__ list, const double* __restrict__ x,
                           const double* __restrict__ y, const double* __restrict__ w, double* __restrict__ partial) {
    __shared__ double red[kThreads / 32];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int q = list[i];
        const double xq = w ? x[q] * w[q] : x[q];
        acc += xq * y[q];
    }
    const double v = warp_sum(acc);
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
// Sum over a warp of float-float values s + e (Knuth's two-sum on the high
// parts, the low parts and both errors added, then Fast2Sum), on the FP32
// pipes; the result is complete in every lane.  Summing in FP64 instead costs
// a conversion, five shuffles and five FP64 adds per lane, which on GB300's
// FP64 rate outweighs the FP32 streaming work of a short grid-stride loop.
__device__ __forceinline__ double ff_warp_sum(float s, float e) {
    float2 v = ff_norm(s, e);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, v.x, o), ol = __shfl_xor_sync(0xffffffffu, v.y, o);
        const float t = __fadd_rn(v.x, oh);
        const float bp = __fsub_rn(t, v.x);
        const float err = __fadd_rn(__fsub_rn(v.x, __fsub_rn(t, bp)), __fsub_rn(oh, bp));
        v = ff_norm(t, __fadd_rn(err, __fadd_rn(v.y, ol)));
    }
    return ff_to_double(v);
}

// One pass of delayed classical Gram-Schmidt (DCGS2): against the finished
// basis Q (j vectors) and the pending vector v, with the new vector w:
//   partial[b][c] = Q_c . v, [j + c] = Q_c . w (c < j), [2j] = v . v, [2j + 1] = v . w
// Columns go in chunks of up to 8 whose size is a compile-time constant, so the
// accumulators stay in registers and no predicated-off column is issued.
// The compact vectors have an even length and stride (a zero pad entry when
// needed), and every thread takes two entries per step with one 16-byte load
// per vector, so twice the bytes are in flight per load instruction.
template <int NC>
__device__ __forceinline__ void dcgs_chunk(long long n2, int j, int c0, const float4* __restrict__ Q, long long ld2,
                                           const float4* __restrict__ v, const float4* __restrict__ w, bool first,
                                           float& as, float& ae, float& ds, float& de, double* __restrict__ partial,
                                           int ldp) {
    __shared__ double red[kThreads / 32][16];
    constexpr int N1 = NC > 0 ? NC : 1;
    float ss[N1], se[N1], cs[N1], ce[N1];
#pragma unroll
    for (int c = 0; c < N1; ++c) ss[c] = se[c] = cs[c] = ce[c] = 0.f;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n2; r += (long long)gridDim.x * blockDim.x) {
        const float4 vv = v[r], ww = w[r];
        if (first) {
            ff_madd(vv.x, vv.y, vv.x, vv.y, as, ae);
            ff_madd(vv.z, vv.w, vv.z, vv.w, as, ae);
            ff_madd(vv.x, vv.y, ww.x, ww.y, ds, de);
            ff_madd(vv.z, vv.w, ww.z, ww.w, ds, de);
        }
        float4 q[N1];
#pragma unroll
        for (int c = 0; c < NC; ++c) q[c] = Q[(c0 + c) * ld2 + r];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            ff_madd(q[c].x, q[c].y, vv.x, vv.y, ss[c], se[c]);
            ff_madd(q[c].z, q[c].w, vv.z, vv.w, ss[c], se[c]);
            ff_madd(q[c].x, q[c].y, ww.x, ww.y, cs[c], ce[c]);
            ff_madd(q[c].z, q[c].w, ww.z, ww.w, cs[c], ce[c]);
        }
    }
    if constexpr (NC > 0) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const double t1 = ff_warp_sum(ss[c], se[c]);
            const double t2 = ff_warp_sum(cs[c], ce[c]);
            if (lane == 0) {
                red[wid][c] = t1;
                red[wid][8 + c] = t2;
            }
        }
        __syncthreads();
        if (threadIdx.x < 2 * NC) {
            const bool isv = threadIdx.x < NC;
            const int c = isv ? threadIdx.x : threadIdx.x - NC;
            double t = 0.0;
            for (int k = 0; k < kThreads / 32; ++k) t += red[k][isv ? c : 8 + c];
            partial[(long long)blockIdx.x * ldp + (isv ? c0 + c : j + c0 + c)] = t;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads, 3) k_ff_dcgs_dots(long long n2, int j, const float4* __restrict__ Q,
                                                              long long ld2, const float4* __restrict__ v,
                                                              const float4* __restrict__ w, double* __restrict__ partial,
                                                              int ldp) {
    __shared__ double red2[kThreads / 32][2];
    float as = 0.f, ae = 0.f, ds = 0.f, de = 0.f;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c0 = 0; c0 < (j > 0 ? j : 1); c0 += 8) {
        const int nc = j > 0 ? min(8, j - c0) : 0;
        const bool first = c0 == 0;
        switch (nc) {
            case 0: dcgs_chunk<0>(n2, j, c0, Q, ld2, v, w, first, as, ae, ds, de, partial, ldp); break;
            case 1: dcgs_chunk<1>(n2, j, c0, Q, ld2, v, w, first, as, ae, ds, de, partial, ldp); break;
            case 2: dcgs_chunk<2>(n2, j, c0, Q, ld2, v, w, first, as, ae, ds, de, partial, ldp); break;
            case 3: dcgs_chunk<3>(n2, j, c0, Q, ld2, v, w, first, as, ae, ds, de, partial, ldp); break;
            case 4: dcgs_chunk<4>(n2, j, c0, Q, ld2, v, w, first, as, ae, ds, de, partial, ldp); break;
            case 5: dcgs_chunk<5>(n2, j, c0, Q, ld2, v, w, first, as, ae, ds, de, partial, ldp); break;
            case 6: dcgs_chunk<6>(n2, j, c0, Q, ld2, v, w, first, as, ae, ds, de, partial, ldp); break;
            case 7: dcgs_chunk<7>(n2, j, c0, Q, ld2, v, w, first, as, ae, ds, de, partial, ldp); break;
            default: dcgs_chunk<8>(n2, j, c0, Q, ld2, v, w, first, as, ae, ds, de, partial, ldp);
        }
    }
    const double ta = ff_warp_sum(as, ae);
    const double td = ff_warp_sum(ds, de);
    if (lane == 0) {
        red2[wid][0] = ta;
        red2[wid][1] = td;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) t += red2[k][threadIdx.x];
        partial[(long long)blockIdx.x * ldp + 2 * j + threadIdx.x] = t;
    }
}

// The update pass of DCGS2, with coef = [s (j), gamma (j), 1/beta, delta]:
//   v <- (v - Q s) / beta   (the pending vector, now finished)
//   out <- w - Q gamma - delta v_old   and the block partial of |out|^2
// Two entries per thread and step, as in the dots pass.
__global__ void k_ff_dcgs_update(long long n2, int j, const float4* __restrict__ Q, long long ld2,
                                 const double* __restrict__ coef, float4* __restrict__ v, const float4* __restrict__ w,
                                 float4* __restrict__ out, double* __restrict__ partial) {
    __shared__ float2 cs[128], cg[128];
    __shared__ float2 rb, dl;
    __shared__ double red[kThreads / 32];
    for (int c = threadIdx.x; c < j; c += blockDim.x) {
        cs[c] = ff_bits(-coef[c]);
        cg[c] = ff_bits(-coef[j + c]);
    }
    if (threadIdx.x == 0) {
        rb = ff_bits(coef[2 * j]);
        dl = ff_bits(-coef[2 * j + 1]);
    }
    __syncthreads();
    float ns = 0.f, ne = 0.f;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n2; r += (long long)gridDim.x * blockDim.x) {
        const float4 vv = v[r], ww = w[r];
        float ts0 = vv.x, te0 = vv.y, ts1 = vv.z, te1 = vv.w;
        float us0 = ww.x, ue0 = ww.y, us1 = ww.z, ue1 = ww.w;
        ff_madd(dl.x, dl.y, vv.x, vv.y, us0, ue0);
        ff_madd(dl.x, dl.y, vv.z, vv.w, us1, ue1);
#pragma unroll 4
        for (int c = 0; c < j; ++c) {
            const float4 q = Q[c * ld2 + r];
            ff_madd(cs[c].x, cs[c].y, q.x, q.y, ts0, te0);
            ff_madd(cs[c].x, cs[c].y, q.z, q.w, ts1, te1);
            ff_madd(cg[c].x, cg[c].y, q.x, q.y, us0, ue0);
            ff_madd(cg[c].x, cg[c].y, q.z, q.w, us1, ue1);
        }
        const float2 t0 = ff_norm(ts0, te0), t1 = ff_norm(ts1, te1);
        float qs0 = 0.f, qe0 = 0.f, qs1 = 0.f, qe1 = 0.f;
        ff_madd(rb.x, rb.y, t0.x, t0.y, qs0, qe0);
        ff_madd(rb.x, rb.y, t1.x, t1.y, qs1, qe1);
        const float2 n0 = ff_norm(qs0, qe0), n1 = ff_norm(qs1, qe1);
        v[r] = make_float4(n0.x, n0.y, n1.x, n1.y);
        const float2 o0 = ff_norm(us0, ue0), o1 = ff_norm(us1, ue1);
        out[r] = make_float4(o0.x, o0.y, o1.x, o1.y);
        ff_madd(o0.x, o0.y, o0.x, o0.y, ns, ne);
        ff_madd(o1.x, o1.y, o1.x, o1.y, ns, ne);
    }
    const double t = ff_warp_sum(ns, ne);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) a += red[k];
        partial[blockIdx.x] = a;
    }
}

// ---- ordered compaction: the indices r < n with flag(x[r]), ascending ----
constexpr int kListChunk = 4096;   // entries per block (256 threads x 16)
template <typename T>
__device__ __forceinline__ bool list_flag(T v) { return v > T(0); }
template <typename T>
__global__ void k_list_count(long long n, const T* __restrict__ x, int* __restrict__ counts) {
    __shared__ int red[kThreads / 32];
    const long long b0 = (long long)blockIdx.x * kListChunk;
    int c = 0;
    for (int k = threadIdx.x; k < kListChunk; k += blockDim.x) {
        const long long r = b0 + k;
        if (r < n && list_flag(x[r])) ++c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        counts[blockIdx.x] = t;
    }
}
// writes the flagged indices of each chunk from offsets[b], in order: the chunk
// goes in rounds of blockDim entries, each round ranked with a block scan
template <typename T>
__global__ void k_list_write(long long n, const T* __restrict__ x, const int* __restrict__ offsets,
                             int* __restrict__ out) {
    __shared__ int wsum[kThreads / 32];
    __shared__ int base;
    const long long b0 = (long long)blockIdx.x * kListChunk;
    if (threadIdx.x == 0) base = offsets[blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k0 = 0; k0 < kListChunk; k0 += blockDim.x) {
        const long long r = b0 + k0 + threadIdx.x;
        const bool f = r < n && list_flag(x[r]);
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        const int before = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        int woff = 0, tot = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            if (w < wid) woff += wsum[w];
            tot += wsum[w];
        }
        if (f) out[base + woff + before] = (int)r;
        __syncthreads();
        if (threadIdx.x == 0) base += tot;
        __syncthreads();
    }
}

// y[i] = split(a x[list[i]])   (gather into a compact float-float vector)
__global__ void k_ff_gather(long long n, const int* __restrict__ list, double a, const double* __restrict__ x,
                            float2* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = ff_bits(a == 1.0 ? x[list[i]] : a * x[list[i]]);
}
// y[list[i]] = a x[i] in storage type T   (scatter from a compact float-float vector)
template <typename T>
__global__ void k_ff_scatter(long long n, const int* __restrict__ list, typename Compute<T>::type a,
                             const float2* __restrict__ x, T* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 v = x[i];
        if constexpr (std::is_same<T, double>::value) y[list[i]] = a * ff_to_double(v);
        else y[list[i]] = to_store<T>(a * __fadd_rn(v.x, v.y));
    }
}

inline int blocks_for(const Domain& d) {
    const long long work = d.tiles ? (long long)d.ntiles : (d.len() + kThreads - 1) / kThreads;
    return (int)std::max<long long>(1, std::min<long long>(work, kMaxBlocks));
}

// Grid of a grid-stride kernel: at most one full wave (the blocks that fit on
// the device at once), so that no partial second wave idles most SMs.
template <typename K>
int blocks_for(const Domain& d, K kernel) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, int> wave;
    int dev = 0;
    DM_CUDA(cudaGetDevice(&dev));
    const auto key = std::make_pair(dev, (const void*)kernel);
    int full;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = wave.find(key);
        if (it == wave.end()) {
            int sms = 0, occ = 0;
            DM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            DM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, 0));
            const int per_sm = std::max(1, std::min(occ, kMaxBlocks / std::max(sms, 1)));
            it = wave.emplace(key, std::max(1, std::min(sms * per_sm, kMaxBlocks))).first;
        }
        full = it->second;
    }
    const long long work = d.tiles ? (long long)d.ntiles : (d.len() + kThreads - 1) / kThreads;
    return (int)std::max<long long>(1, std::min<long long>(work, full));
}

}  // namespace

void reducer_init(Reducer& r, int max_cols) {
    r.cap_blocks = kMaxBlocks;
    r.max_cols = max_cols;
    note_allocation();
    DM_CUDA(cudaMalloc(&r.partial, sizeof(double) * (size_t)r.cap_blocks * max_cols));
    note_allocation();
    DM_CUDA(cudaMalloc(&r.result, sizeof(double) * (size_t)max_cols));
    note_allocation();
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
    const int nb = blocks_for(d, k_mdot_partial);
    launch_b("k_mdot_partial", 8.0 * d.live() * (m + 1 + (w ? 1 : 0)), k_mdot_partial, nb, kThreads, 0, s, d, m, V,
             ld, x, w, red.partial, red.max_cols, 0);
    launch("k_mdot_final", k_mdot_final, (m + 7) / 8, 256, 0, s, nb, m, red.partial, red.max_cols, red.result);
    DM_CUDA(cudaMemcpyAsync(red.host, red.result, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < m; ++c) host_out[c] = red.host[c];
}

double dot_list(Reducer& red, long long n, const int* list, const double* x, const double* y, const double* w,
                cudaStream_t s) {
    if (n <= 0) return 0.0;
    const int nb = (int)std::max<long long>(1, std::min<long long>((n + kThreads - 1) / kThreads, kMaxBlocks));
    launch_b("k_dot_list", (w ? 28.0 : 20.0) * (double)n, k_dot_list, nb, kThreads, 0, s, n, list, x, y, w,
             red.partial);
    launch("k_mdot_final", k_mdot_final, 1, 256, 0, s, nb, 1, red.partial, 1, red.result);
    DM_CUDA(cudaMemcpyAsync(red.host, red.result, sizeof(double), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    return red.host[0];
}

void mdot_self(Reducer& red, const Domain& d, int m, const double* V, long long ld, const double* x, const double* w,
               double* host_out, double* self_out, cudaStream_t s) {
    DM_REQUIRE(m >= 1 && m + 1 <= red.max_cols, DM_ERR_INVALID_ARG, "mdot: too many columns");
    const int nb = blocks_for(d, k_mdot_partial);
    launch_b("k_mdot_partial", 8.0 * d.live() * (m + 1 + (w ? 1 : 0)), k_mdot_partial, nb, kThreads, 0, s, d, m, V,
             ld, x, w, red.partial, red.max_cols, 1);
    launch("k_mdot_final", k_mdot_final, (m + 1 + 7) / 8, 256, 0, s, nb, m + 1, red.partial, red.max_cols, red.result);
    DM_CUDA(cudaMemcpyAsync(red.host, red.result, sizeof(double) * (m + 1), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < m; ++c) host_out[c] = red.host[c];
    *self_out = red.host[m];
}

double maxpy_norm(Reducer& red, const Domain& d, int m, const double* V, long long ld, double* x, const double* w,
                  cudaStream_t s) {
    DM_REQUIRE(m >= 1 && m <= 128 && m <= red.max_cols, DM_ERR_INVALID_ARG, "maxpy: too many columns");
    const int nb = blocks_for(d, k_maxpy_norm);
    // h = red.result (written by the preceding mdot on this stream); partials in a separate stripe
    double* part = red.partial + (size_t)red.cap_blocks * (red.max_cols - 1);
    launch_b("k_maxpy_norm", 8.0 * d.live() * (m + 2 + (w ? 1 : 0)), k_maxpy_norm, nb, kThreads, 0, s, d, m, V, ld,
             red.result, x, w, part);
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
    launch_b("k_maxpy", 8.0 * d.live() * (m + 2), k_maxpy, blocks_for(d, k_maxpy), kThreads, 0, s, d, m, V, ld,
             red.result, x);
}

template <typename T>
int list_flagged(long long n, const T* x, DBuf<int>& out, cudaStream_t s) {
    const int nb = (int)std::max<long long>(1, (n + kListChunk - 1) / kListChunk);
    DBuf<int> counts(nb, false), offsets(nb, false);
    launch("k_list_count", k_list_count<T>, nb, kThreads, 0, s, n, x, counts.get());
    std::vector<int> h(nb);
    DM_CUDA(cudaMemcpyAsync(h.data(), counts.get(), sizeof(int) * nb, cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    long long tot = 0;
    for (int b = 0; b < nb; ++b) {
        const int c = h[b];
        h[b] = (int)tot;
        tot += c;
    }
    DM_REQUIRE(tot < (1ll << 31), DM_ERR_INVALID_ARG, "list too long");
    out.alloc((size_t)std::max<long long>(tot, 1), false);
    DM_CUDA(cudaMemcpyAsync(offsets.get(), h.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s));
    launch("k_list_write", k_list_write<T>, nb, kThreads, 0, s, n, x, (const int*)offsets.get(), out.get());
    DM_CUDA(cudaStreamSynchronize(s));
    return (int)tot;
}
template int list_flagged<double>(long long, const double*, DBuf<int>&, cudaStream_t);
template int list_flagged<unsigned char>(long long, const unsigned char*, DBuf<int>&, cudaStream_t);

void ff_gather(long long n, const int* list, double a, const double* x, float2* y, cudaStream_t s) {
    const int nb = (int)std::max<long long>(1, std::min<long long>((n + kThreads - 1) / kThreads, kMaxBlocks));
    launch_b("k_ff_gather", 20.0 * n, k_ff_gather, nb, kThreads, 0, s, n, list, a, x, y);
}
template <typename T>
void ff_scatter(long long n, const int* list, double a, const float2* x, T* y, cudaStream_t s) {
    const int nb = (int)std::max<long long>(1, std::min<long long>((n + kThreads - 1) / kThreads, kMaxBlocks));
    launch_b("k_ff_scatter", (12.0 + sizeof(T)) * n, k_ff_scatter<T>, nb, kThreads, 0, s, n, list,
             (typename Compute<T>::type)a, x, y);
}
template void ff_scatter<double>(long long, const int*, double, const float2*, double*, cudaStream_t);
template void ff_scatter<float>(long long, const int*, double, const float2*, float*, cudaStream_t);
template void ff_scatter<__nv_bfloat16>(long long, const int*, double, const float2*, __nv_bfloat16*, cudaStream_t);

// blocks of the two-entry DCGS passes: enough for one wave of pairs
template <typename K>
int pair_blocks(long long n2, K kernel) {
    int per_sm = 0;
    DM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0));
    const long long need = (n2 + kThreads - 1) / kThreads;
    return (int)std::max<long long>(1, std::min<long long>(need, 152ll * std::max(per_sm, 1)));
}

void dcgs_dots(Reducer& red, const Domain& d, int j, const float2* Q, long long ld, const float2* v, const float2* w,
               double* host_out, cudaStream_t s) {
    const int m = 2 * j + 2;
    DM_REQUIRE(j >= 0 && j <= 120 && m < red.max_cols, DM_ERR_INVALID_ARG, "dcgs: too many columns");
    DM_REQUIRE(d.tiles == nullptr && d.len() % 2 == 0 && ld % 2 == 0, DM_ERR_INVALID_ARG,
               "dcgs: compact vectors need an even length and stride");
    const long long n2 = d.len() / 2;
    const int nb = std::min(pair_blocks(n2, k_ff_dcgs_dots), red.cap_blocks);
    // j finished basis vectors, v and w: float-float, 8 bytes an entry
    launch_b("k_ff_dcgs_dots", 8.0 * d.live() * (j + 2), k_ff_dcgs_dots, nb, kThreads, 0, s, n2, j,
             reinterpret_cast<const float4*>(Q), ld / 2, reinterpret_cast<const float4*>(v),
             reinterpret_cast<const float4*>(w), red.partial, red.max_cols);
    launch("k_mdot_final", k_mdot_final, (m + 7) / 8, 256, 0, s, nb, m, red.partial, red.max_cols, red.result);
    DM_CUDA(cudaMemcpyAsync(red.host, red.result, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < m; ++c) host_out[c] = red.host[c];
}

double dcgs_update(Reducer& red, const Domain& d, int j, const float2* Q, long long ld, const double* coef_host,
                   float2* v, const float2* w, float2* out, cudaStream_t s) {
    DM_REQUIRE(j >= 0 && j <= 120 && 2 * j + 2 <= red.max_cols, DM_ERR_INVALID_ARG, "dcgs: too many columns");
    // coefficients through the pinned host buffer (the preceding dots have synchronised the stream)
    for (int c = 0; c < 2 * j + 2; ++c) red.host[c] = coef_host[c];
    DM_CUDA(cudaMemcpyAsync(red.result, red.host, sizeof(double) * (2 * j + 2), cudaMemcpyHostToDevice, s));
    DM_REQUIRE(d.tiles == nullptr && d.len() % 2 == 0 && ld % 2 == 0, DM_ERR_INVALID_ARG,
               "dcgs: compact vectors need an even length and stride");
    const long long n2 = d.len() / 2;
    const int nb = std::min(pair_blocks(n2, k_ff_dcgs_update), red.cap_blocks);
    double* part = red.partial + (size_t)red.cap_blocks * (red.max_cols - 1);
    // reads Q (j vectors), v and w; writes v and out
    launch_b("k_ff_dcgs_update", 8.0 * d.live() * (j + 4), k_ff_dcgs_update, nb, kThreads, 0, s, n2, j,
             reinterpret_cast<const float4*>(Q), ld / 2, (const double*)red.result, reinterpret_cast<float4*>(v),
             reinterpret_cast<const float4*>(w), reinterpret_cast<float4*>(out), part);
    launch("k_mdot_final", k_mdot_final, 1, 256, 0, s, nb, 1, part, 1, red.result + red.max_cols - 1);
    DM_CUDA(cudaMemcpyAsync(red.host, red.result + red.max_cols - 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    return red.host[0];
}
void vgemm(const Domain& d, int m, int p, const double* V, long long ld, const double* Y_dev, int ldy, double* out,
           long long ldo, cudaStream_t s) {
    const size_t sm = sizeof(double) * (size_t)m * p;
    DM_REQUIRE(sm <= 48 * 1024, DM_ERR_INVALID_ARG, "vgemm: basis too large");
    launch_b("k_vgemm", 8.0 * d.live() * (m + p), k_vgemm, blocks_for(d, k_vgemm), kThreads, sm, s, d, m, p, V, ld,
             Y_dev, ldy, out, ldo);
}

void axpby(const Domain& d, double a, const double* x, double b, double* y, cudaStream_t s) {
    launch_b("k_axpby", 24.0 * d.live(), k_axpby, blocks_for(d, k_axpby), kThreads, 0, s, d, a, x, b, y);
}
void scale_copy(const Domain& d, double a, const double* x, double* y, cudaStream_t s) {
    if (x == y)
        launch_b("k_scale_inplace", 16.0 * d.live(), k_scale_inplace, blocks_for(d, k_scale_inplace), kThreads, 0, s,
                 d, a, y);
    else
        launch_b("k_scale_copy", 16.0 * d.live(), k_scale_copy, blocks_for(d, k_scale_copy), kThreads, 0, s, d, a, x,
                 y);
}
void hadamard(const Domain& d, const double* a, const double* x, double* y, cudaStream_t s) {
    launch_b("k_hadamard", 24.0 * d.live(), k_hadamard, blocks_for(d, k_hadamard), kThreads, 0, s, d, a, x, y);
}
template <typename TD, typename TS>
void convert(const Domain& d, const TS* x, TD* y, cudaStream_t s) {
    launch_b("k_convert", (double)(sizeof(TD) + sizeof(TS)) * d.live(), k_convert<TD, TS>, blocks_for(d, k_convert<TD, TS>),
             kThreads, 0, s, d, x, y);
}
template <typename TD>
void convert_coeff(long long n, const double* x, TD* y, cudaStream_t s) {
    const int b = (int)std::max<long long>(1, std::min<long long>((n + kThreads - 1) / kThreads, kMaxBlocks));
    launch("k_convert_coeff", k_convert_coeff<TD>, b, kThreads, 0, s, n, x, y);
}
void fill_random(const Domain& d, unsigned long long seed, const double* mask, double* x, cudaStream_t s) {
    launch("k_fill_random", k_fill_random, blocks_for(d, k_fill_random), kThreads, 0, s, d, seed, mask, x);
}
void zero(void* p, size_t bytes, cudaStream_t s) { DM_CUDA(cudaMemsetAsync(p, 0, bytes, s)); }

template void convert<float, double>(const Domain&, const double*, float*, cudaStream_t);
template void convert<double, float>(const Domain&, const float*, double*, cudaStream_t);
template void convert<__nv_bfloat16, double>(const Domain&, const double*, __nv_bfloat16*, cudaStream_t);
template void convert<double, __nv_bfloat16>(const Domain&, const __nv_bfloat16*, double*, cudaStream_t);
template void convert<double, double>(const Domain&, const double*, double*, cudaStream_t);
template void convert_coeff<float>(long long, const double*, float*, cudaStream_t);

}  // namespace dm
