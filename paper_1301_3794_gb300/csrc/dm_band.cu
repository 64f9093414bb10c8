// Cut-cell band smoother: a restricted additive Schwarz step on the band faces.
//
// The band holds the open faces next to a cell within one cell of a cut cell
// (0 < V < 1).  It is covered by bricks of b^3 nodes (a face belongs to the
// node at its lower corner).  The subdomain of a brick is every band face whose
// node lies within one node of the brick; the brick owns the faces whose node
// lies inside it.  From r0 = f - (K - sigma A) x, each subdomain runs `sweeps`
// damped Jacobi sweeps d <- d + omega D^-1 (r0 - K_SS d) from d = 0 on its own
// rows (couplings to faces outside the subdomain stay frozen), and x takes d
// on the owned faces.  With one brick covering the grid this is plain
// band-restricted Jacobi.
//
// One thread block per subdomain.  The correction d lives in shared memory on
// the subdomain's local box of nodes (all three components, zero wherever the
// subdomain has no row), so a row's couplings are reached at fixed offsets:
// the 15 slots of band_slot.  Each thread keeps the coefficients of its rows in
// registers, so every sweep after the first touches only registers and shared
// memory, with one block barrier per sweep and none across the grid.
#include <algorithm>
#include <vector>

#include "dm_common.cuh"

namespace dm {

namespace {

// Couplings of a row in the subdomain's local box: component c at local node
// n (index within one component's box), box strides st = {1, lx, lx ly}, l3
// nodes per component.  The 15 slots of band_slot, in order, are
//   same component:   n, n -/+ 1, n -/+ lx, n -/+ lx ly;
//   component c + k (k = 1, 2), its stride sk = st[(c + k) % 3]:
//     m, m + sk, m + sc, m + sc + sk  with m = n - sc (sc = st[c]) in that component.
struct RowAddr {
    int b0, b1, b2;   // n, and m in components c + 1 and c + 2 (offsets into the box)
    int sc, s1, s2;
};
__device__ __forceinline__ RowAddr row_addr(int p, int l3, int lx, int lxy) {
    RowAddr a;
    const int c = p / l3, n = p - c * l3;
    const int st[3] = {1, lx, lxy};
    const int c1 = c == 2 ? 0 : c + 1, c2 = c == 0 ? 2 : c - 1;
    a.sc = st[c];
    a.s1 = st[c1];
    a.s2 = st[c2];
    a.b0 = p;
    a.b1 = c1 * l3 + n - a.sc;
    a.b2 = c2 * l3 + n - a.sc;
    return a;
}
// `self` is the row's own entry d[a.b0] (kept in a register by the sweeps)
template <typename C>
__device__ __forceinline__ C row_dot(const C* v, C self, const C* d, const RowAddr& a, int lx, int lxy) {
    C acc = v[0] * self;
    acc += v[1] * d[a.b0 - 1] + v[2] * d[a.b0 + 1];
    acc += v[3] * d[a.b0 - lx] + v[4] * d[a.b0 + lx];
    acc += v[5] * d[a.b0 - lxy] + v[6] * d[a.b0 + lxy];
    acc += v[7] * d[a.b1] + v[8] * d[a.b1 + a.s1] + v[9] * d[a.b1 + a.sc] + v[10] * d[a.b1 + a.sc + a.s1];
    acc += v[11] * d[a.b2] + v[12] * d[a.b2 + a.s2] + v[13] * d[a.b2 + a.sc] + v[14] * d[a.b2 + a.sc + a.s2];
    return acc;
}

// The default brick (8 nodes) uses one fixed local box for every subdomain:
// nodes B b - 2 .. B b + 9 on each axis (12 nodes; x padded to 13 to spread
// shared-memory banks), so every coupling offset is a compile-time constant.
constexpr int kFixedBrick = 8, kFX = 13, kFY = 12, kFZ = 12, kFXY = kFX * kFY, kF3 = kFXY * kFZ;

template <typename C, int c>
__device__ __forceinline__ C row_dot_fixed(const C* v, C self, const C* d, int p) {
    constexpr int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
    constexpr int sc = c == 0 ? 1 : (c == 1 ? kFX : kFXY);
    constexpr int s1 = c1 == 0 ? 1 : (c1 == 1 ? kFX : kFXY);
    constexpr int s2 = c2 == 0 ? 1 : (c2 == 1 ? kFX : kFXY);
    constexpr int o1 = (c1 - c) * kF3 - sc, o2 = (c2 - c) * kF3 - sc;
    const C* q = d + p;
    C acc = v[0] * self;
    acc += v[1] * q[-1] + v[2] * q[1];
    acc += v[3] * q[-kFX] + v[4] * q[kFX];
    acc += v[5] * q[-kFXY] + v[6] * q[kFXY];
    acc += v[7] * q[o1] + v[8] * q[o1 + s1] + v[9] * q[o1 + sc] + v[10] * q[o1 + sc + s1];
    acc += v[11] * q[o2] + v[12] * q[o2 + s2] + v[13] * q[o2 + sc] + v[14] * q[o2 + sc + s2];
    return acc;
}
template <typename C>
__device__ __forceinline__ C row_dot_fixed(int c, const C* v, C self, const C* d, int p) {
    return c == 0 ? row_dot_fixed<C, 0>(v, self, d, p)
                  : (c == 1 ? row_dot_fixed<C, 1>(v, self, d, p) : row_dot_fixed<C, 2>(v, self, d, p));
}

// R > 0: each thread owns up to R rows (row r = threadIdx.x + k blockDim.x) with
// their coefficients and addresses in registers.  R == 0: any row count; r0
// and omega/D in shared memory and the coefficients re-read on every sweep.
// Block b handles subdomain sub0 + b.
template <typename T, typename TC, int R, int NT, bool FIXED>
__global__ void __launch_bounds__(NT)
    k_band_schwarz(int sub0, const int* __restrict__ off, const int* __restrict__ copy, const int* __restrict__ pos,
                   const int* __restrict__ dims, const int* __restrict__ org, const TC* __restrict__ vals, int ncopies,
                   const int* __restrict__ band, const TC* __restrict__ invD, const T* __restrict__ f,
                   const T* __restrict__ x, double* __restrict__ u, typename Compute<T>::type om, int sweeps, Grid3 g,
                   int maxbox, int maxrows) {
    using C = typename Compute<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* const buf0 = reinterpret_cast<C*>(smem_raw);
    C* const buf1 = buf0 + maxbox;
    C* s_r0 = buf1 + maxbox;          // R == 0 only
    C* s_w = s_r0 + maxrows;
    const int sd = sub0 + blockIdx.x;
    const int b0 = off[sd];
    const int nr = off[sd + 1] - b0;
    const int dm = dims[sd];
    const int lx = FIXED ? kFX : dm & 1023, ly = FIXED ? kFY : (dm >> 10) & 1023, lz = FIXED ? kFZ : dm >> 20;
    const int lxy = lx * ly, l3 = lxy * lz;
    // x over the local box (nodes org + local coordinates; outside the padded
    // grid's -1 .. n+1 it is zero), so that the start residuals read it from
    // shared memory at the rows' slot offsets: one coalesced pass over the box
    // instead of 15 scattered loads per row
    {
        const int ox = org[3 * sd], oy = org[3 * sd + 1], oz = org[3 * sd + 2];
        for (int k = threadIdx.x; k < 3 * l3; k += blockDim.x) {
            const int comp = k / l3, n = k - comp * l3;
            const int lk = n / lxy, rem = n - lk * lxy;
            const int lj = rem / lx, li = rem - lj * lx;
            const int i = ox + li, j = oy + lj, kk = oz + lk;
            const bool in = i >= -1 && j >= -1 && kk >= -1 && i <= g.nx + 1 && j <= g.ny + 1 && kk <= g.nz + 1;
            buf0[k] = C(0);
            buf1[k] = in ? (C)to_c(x[(size_t)comp * g.np + g.idx(i, j, kk)]) : C(0);
        }
    }
    __syncthreads();
    constexpr int RR = R > 0 ? R : 1;
    C v[RR][kBandSlots];
    C r0[RR], w[RR], dself[RR];   // dself: the row's current correction (R > 0)
    RowAddr ad[RR];
    int cm[RR];
    // residual of the full row at the start values, and the first sweep from d = 0
    auto start_row = [&](int r, C* ve, C& rr, C& ww) {
        const int ct = copy[b0 + r];
        if (ct == kDummyCopy) {   // an empty lane of a warp group: no row, no loads
#pragma unroll
            for (int e = 0; e < kBandSlots; ++e) ve[e] = C(0);
            rr = C(0);
            ww = C(0);
            return;
        }
        const int t = ct >= 0 ? ct : -1 - ct;
        const int q = band[t];
        const int ps = pos[b0 + r];
#pragma unroll
        for (int e = 0; e < kBandSlots; ++e) ve[e] = (C)vals[(size_t)e * ncopies + b0 + r];
        const C acc = FIXED ? row_dot_fixed(ps / l3, ve, buf1[ps], buf1, ps)
                            : row_dot(ve, buf1[ps], buf1, row_addr(ps, l3, lx, lxy), lx, lxy);
        rr = (C)to_c(f[q]) - acc;
        ww = om * (C)invD[q];
        buf0[ps] = ww * rr;
    };
    if constexpr (R > 0) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int r = threadIdx.x + k * blockDim.x;
            cm[k] = -1;
            if (r < nr) {
                start_row(r, v[k], r0[k], w[k]);
                dself[k] = w[k] * r0[k];
                const int ps = pos[b0 + r];
                if (ps >= 0) {
                    ad[k] = row_addr(ps, l3, lx, lxy);
                    cm[k] = ps / l3;
                }
            }
        }
    } else {
        for (int r = threadIdx.x; r < nr; r += blockDim.x) start_row(r, v[0], s_r0[r], s_w[r]);
    }
    __syncthreads();
    // buf1 becomes the second correction buffer: zero outside the rows
    for (int k = threadIdx.x; k < 3 * l3; k += blockDim.x) buf1[k] = C(0);
    __syncthreads();
    C* dc = buf0;
    C* dn = buf1;
    for (int s = 1; s < sweeps; ++s) {
        if constexpr (R > 0) {
#pragma unroll
            for (int k = 0; k < RR; ++k) {
                const int r = threadIdx.x + k * blockDim.x;
                if (r < nr && cm[k] >= 0) {
                    const C acc = FIXED ? row_dot_fixed(cm[k], v[k], dself[k], dc, ad[k].b0)
                                        : row_dot(v[k], dself[k], dc, ad[k], lx, lxy);
                    dself[k] = dself[k] + w[k] * (r0[k] - acc);
                    dn[ad[k].b0] = dself[k];
                }
            }
        } else {
            for (int r = threadIdx.x; r < nr; r += blockDim.x) {
                const int ps = pos[b0 + r];
                if (ps < 0) continue;
                const RowAddr a = row_addr(ps, l3, lx, lxy);
                C ve[kBandSlots];
#pragma unroll
                for (int e = 0; e < kBandSlots; ++e) ve[e] = (C)vals[(size_t)e * ncopies + b0 + r];
                const C self = dc[a.b0];
                dn[a.b0] = self + s_w[r] * (s_r0[r] - row_dot(ve, self, dc, a, lx, lxy));
            }
        }
        __syncthreads();
        C* const tmp = dc;
        dc = dn;
        dn = tmp;
    }
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        const int ct = copy[b0 + r];
        if (ct >= 0) u[ct] = (double)dc[pos[b0 + r]];
    }
}

template <typename T>
__global__ void k_band_add(const int* __restrict__ band, int nband, const double* __restrict__ u,
                           T* __restrict__ x) {
    using C = typename Compute<T>::type;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nband) return;
    const int q = band[t];
    x[q] = to_store<T>((C)to_c(x[q]) + (C)u[t]);
}

__global__ void k_band_copy_vals(const int* __restrict__ copy, int ncopies, const double* __restrict__ band_vals,
                                 int nband, double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncopies) return;
    const int ct = copy[c];
    if (ct == kDummyCopy) {
        for (int e = 0; e < kBandSlots; ++e) out[(size_t)e * ncopies + c] = 0.0;
        return;
    }
    const int t = ct >= 0 ? ct : -1 - ct;
    for (int e = 0; e < kBandSlots; ++e) out[(size_t)e * ncopies + c] = band_vals[(size_t)e * nband + t];
}

template <typename T>
size_t schwarz_smem(int maxbox, int maxrows, int R) {
    using C = typename Compute<T>::type;
    return sizeof(C) * (2 * (size_t)maxbox + (R == 0 ? 2 * (size_t)maxrows : 0));
}

}  // namespace

// Size classes of subdomains (rows): each class is launched with its own
// block size and rows per thread, so that small subdomains are not held to the
// register and thread budget of the largest.
// levels with at most this many subdomains are smoothed in a single launch
constexpr int kSingleLaunchSubdomains = 304;

int schwarz_class(int rows) {
    return rows <= 256 ? 0 : (rows <= 512 ? 1 : (rows <= 1024 ? 2 : (rows <= 2048 ? 3 : 4)));
}

namespace {

}  // namespace

void band_schwarz_setup(const Grid3& g, const int* band_dev, int nband, int brick, SchwarzLayout& out,
                        cudaStream_t s) {
    DM_REQUIRE(brick >= 1, DM_ERR_INVALID_ARG, "band brick must be >= 1 node");
    out = SchwarzLayout{};
    if (nband <= 0) return;
    std::vector<int> band(nband);
    DM_CUDA(cudaMemcpyAsync(band.data(), band_dev, sizeof(int) * nband, cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));

    // node (i, j, k) and component of every band face: q = c np + off0 + i + sx (j + sy k)
    const int n[3] = {g.nx, g.ny, g.nz};
    const int nb[3] = {(g.nx + brick) / brick, (g.ny + brick) / brick, (g.nz + brick) / brick};
    std::vector<int> node((size_t)3 * nband);
    std::vector<char> owner((size_t)nb[0] * nb[1] * nb[2], 0);
    auto key = [&](int bx, int by, int bz) { return ((long long)bz * nb[1] + by) * nb[0] + bx; };
    for (int t = 0; t < nband; ++t) {
        const int q = band[t];
        const int r = q % g.np - g.off0;
        const int k = r / g.sxy, rem = r - k * g.sxy;
        const int j = rem / g.sx, i = rem - j * g.sx;
        node[3 * t] = i;
        node[3 * t + 1] = j;
        node[3 * t + 2] = k;
        owner[key(i / brick, j / brick, k / brick)] = 1;
    }
    // copies (brick, face): brick B holds node P when B b - 1 <= P <= B b + b on every axis,
    // i.e. ceil(P / b) - 1 <= B <= floor((P + 1) / b)
    struct Copy {
        long long brick;
        int q, t;
        bool owned;
    };
    // grouped by brick with a counting sort (two passes over the faces), then
    // each brick's copies sorted by face index: the order of one sort by
    // (brick, face) at a fraction of its cost
    const size_t nbk = (size_t)nb[0] * nb[1] * nb[2];
    auto each_copy = [&](auto&& visit) {
        for (int t = 0; t < nband; ++t) {
            int lo[3], hi[3], own[3];
            for (int a = 0; a < 3; ++a) {
                const int P = node[3 * t + a];
                own[a] = P / brick;
                lo[a] = std::max((P + brick - 1) / brick - 1, 0);
                hi[a] = std::min((P + 1) / brick, nb[a] - 1);
            }
            for (int bz = lo[2]; bz <= hi[2]; ++bz)
                for (int by = lo[1]; by <= hi[1]; ++by)
                    for (int bx = lo[0]; bx <= hi[0]; ++bx) {
                        const long long kb = key(bx, by, bz);
                        if (owner[kb]) visit(kb, t, bx == own[0] && by == own[1] && bz == own[2]);
                    }
        }
    };
    std::vector<long long> start(nbk + 1, 0);
    each_copy([&](long long kb, int, bool) { ++start[kb + 1]; });
    for (size_t b = 0; b < nbk; ++b) start[b + 1] += start[b];
    std::vector<Copy> cp((size_t)start[nbk]);
    {
        std::vector<long long> fill(start.begin(), start.end() - 1);
        each_copy([&](long long kb, int t, bool owned) { cp[(size_t)fill[kb]++] = Copy{kb, band[t], t, owned}; });
    }
    for (size_t b = 0; b < nbk; ++b)
        std::sort(cp.begin() + start[b], cp.begin() + start[b + 1],
                  [](const Copy& a, const Copy& c) { return a.q < c.q; });
    const int nc = (int)cp.size();
    // subdomains (runs of one brick), emitted class by class
    std::vector<std::pair<int, int>> runs;
    for (int c0 = 0; c0 < nc;) {
        int c1 = c0;
        while (c1 < nc && cp[c1].brick == cp[c0].brick) ++c1;
        runs.push_back({c0, c1});
        c0 = c1;
    }
    // slots of a run: its rows per component rounded up to whole warp groups
    auto slots_of = [&](const std::pair<int, int>& r) {
        int n[3] = {0, 0, 0};
        for (int c = r.first; c < r.second; ++c) ++n[cp[c].q / g.np];
        return 32 * ((n[0] + 31) / 32 + (n[1] + 31) / 32 + (n[2] + 31) / 32);
    };
    std::vector<int> run_slots;
    run_slots.reserve(runs.size());
    for (const auto& r : runs) run_slots.push_back(slots_of(r));
    std::vector<int> order(runs.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return schwarz_class(run_slots[a]) < schwarz_class(run_slots[b]);
    });
    {
        std::vector<std::pair<int, int>> sorted;
        sorted.reserve(runs.size());
        for (int i : order) sorted.push_back(runs[i]);
        runs.swap(sorted);
        std::vector<int> rs;
        rs.reserve(order.size());
        for (int i : order) rs.push_back(run_slots[i]);
        run_slots.swap(rs);
    }
    for (int k = 0; k < kSchwarzClasses; ++k) {
        out.cls_first[k] = out.cls_count[k] = 0;
        out.cls_copies[k] = out.cls_owned[k] = 0;
    }
    out.copy.reserve((size_t)nc + 96 * runs.size());
    out.pos.reserve((size_t)nc + 96 * runs.size());
    for (size_t rI = 0; rI < runs.size(); ++rI) {
        const int c0 = runs[rI].first, c1 = runs[rI].second;
        const int cl = schwarz_class(run_slots[rI]);
        if (out.cls_count[cl] == 0) out.cls_first[cl] = (int)rI;
        ++out.cls_count[cl];
        const long long kb = cp[c0].brick;
        const int B[3] = {(int)(kb % nb[0]), (int)((kb / nb[0]) % nb[1]), (int)(kb / ((long long)nb[0] * nb[1]))};
        // local box: the subdomain's nodes and their neighbours (within the
        // padded grid; the default brick uses the fixed, unclipped box)
        int lo[3], l[3];
        for (int a = 0; a < 3; ++a) {
            if (brick == kFixedBrick) {
                lo[a] = B[a] * brick - 2;
                l[a] = a == 0 ? kFX : (a == 1 ? kFY : kFZ);
            } else {
                lo[a] = std::max(B[a] * brick - 2, -1);
                const int hi = std::min(B[a] * brick + brick + 1, n[a] + 1);
                l[a] = hi - lo[a] + 1;
            }
        }
        DM_REQUIRE(l[0] < 1024 && l[1] < 1024 && l[2] < 1024, DM_ERR_INVALID_ARG, "band brick too large");
        out.off.push_back((int)out.copy.size());
        out.dims.push_back(l[0] | (l[1] << 10) | (l[2] << 20));
        out.org.insert(out.org.end(), {lo[0], lo[1], lo[2]});
        out.maxbox = std::max(out.maxbox, 3 * l[0] * l[1] * l[2]);
        out.cls_copies[cl] += c1 - c0;
        // Rows are laid out in warp groups of 32 slots.  Per component, the rows
        // are sorted by their shared-memory bank (box position mod 32) and dealt
        // round-robin over the component's ceil(n / 32) groups, so the lanes of
        // a warp mostly sit in distinct banks; every slot offset is the same for
        // the rows of one component, so each of the 15 loads of a sweep is then
        // (nearly) free of bank conflicts.  Unfilled slots are empty lanes.
        std::vector<std::pair<int, int>> rows[3];   // (position, copy code) per component
        for (int c = c0; c < c1; ++c) {
            const int t = cp[c].t;
            const int comp = cp[c].q / g.np;
            if (cp[c].owned) ++out.cls_owned[cl];
            const int li = node[3 * t] - lo[0], lj = node[3 * t + 1] - lo[1], lk = node[3 * t + 2] - lo[2];
            rows[comp].push_back({((comp * l[2] + lk) * l[1] + lj) * l[0] + li, cp[c].owned ? t : -1 - t});
        }
        for (int comp = 0; comp < 3; ++comp) {
            std::vector<std::pair<int, int>>& rc = rows[comp];
            const int n = (int)rc.size();
            if (n == 0) continue;
            std::stable_sort(rc.begin(), rc.end(), [](const std::pair<int, int>& a, const std::pair<int, int>& b) {
                return (a.first & 31) < (b.first & 31);
            });
            const int ng = (n + 31) / 32;
            const size_t base = out.copy.size();
            out.copy.resize(base + 32 * (size_t)ng, kDummyCopy);
            out.pos.resize(base + 32 * (size_t)ng, -1);
            for (int i = 0; i < n; ++i) {
                const size_t slot = base + (size_t)(i % ng) * 32 + i / ng;
                out.pos[slot] = rc[i].first;
                out.copy[slot] = rc[i].second;
            }
        }
        out.maxrows = std::max(out.maxrows, (int)out.copy.size() - out.off.back());
    }
    out.off.push_back((int)out.copy.size());
    out.fixed = brick == kFixedBrick;
}

void band_copy_vals(const int* copy, int ncopies, const double* band_vals, int nband, double* out, cudaStream_t s) {
    if (ncopies <= 0) return;
    launch("k_band_copy_vals", k_band_copy_vals, (ncopies + 255) / 256, 256, 0, s, copy, ncopies, band_vals, nband,
           out);
}

// rows per thread and block size of a class (R = 0: the shared-memory variant;
// FP64 rows hold twice the registers, so FP64 stops at R = 2)
template <typename T>
void class_shape(int cl, int& R, int& nt) {
    const bool wide = sizeof(typename Compute<T>::type) == 8;
    switch (cl) {
        case 0: R = 1; nt = 256; break;
        case 1: R = 1; nt = 512; break;
        case 2: R = 2; nt = 512; break;
        case 3: R = wide ? 0 : 4; nt = 512; break;
        default: R = 0; nt = 512;
    }
}

template <typename T, typename TC>
void band_schwarz(const BandSchwarz<TC>& bs, const TC* invD, const Grid3& g, const int* band, int nband, const T* f,
                  T* x, double* u, double omega, int sweeps, bool fine, cudaStream_t s0, const Fork* fk) {
    if (nband <= 0 || bs.nsub <= 0 || sweeps <= 0) return;
    const char* name = stencil_name("band_schwarz", prec_index<T>(), ST_JACOBI, fine);
    // a level whose subdomains fit in one wave goes in a single launch shaped for
    // its largest class; larger levels launch each class with its own shape
    int top = 0;
    for (int cl = 0; cl < kSchwarzClasses; ++cl)
        if (bs.cls_count[cl] > 0) top = cl;
    const bool single = bs.nsub <= kSingleLaunchSubdomains;
    // classes launched here, and the stream each takes
    int nl = 0;
    for (int cl = 0; cl < kSchwarzClasses; ++cl)
        if (bs.cls_count[cl] > 0 && !(single && cl != top)) ++nl;
    const bool forked = fk && fk->naux > 0 && nl > 1;
    if (forked) {
        DM_CUDA(cudaEventRecord(fk->fork, s0));
        for (int a = 0; a < std::min(nl - 1, fk->naux); ++a) DM_CUDA(cudaStreamWaitEvent(fk->aux[a], fk->fork, 0));
    }
    int li = 0;
    for (int cl = 0; cl < kSchwarzClasses; ++cl) {
        if (bs.cls_count[cl] == 0 || (single && cl != top)) continue;
        const int ai = li++;   // the first class stays on s0
        cudaStream_t s = (forked && ai > 0 && ai - 1 < fk->naux) ? fk->aux[ai - 1] : s0;
        int R, nt;
        class_shape<T>(single ? top : cl, R, nt);
        const int first = single ? 0 : bs.cls_first[cl];
        const int count = single ? bs.nsub : bs.cls_count[cl];
        const size_t smem = schwarz_smem<T>(bs.maxbox, bs.maxrows, R);
        // bytes: per row copy its 15 coefficients, copy and pos words, and the
        // row's x, f and 1/D (the slot gathers of x hit the row's neighbours,
        // which are other copies' rows); per owned copy the correction u
        long long copies = 0, owned = 0;
        for (int k = 0; k < kSchwarzClasses; ++k)
            if (single || k == cl) {
                copies += bs.cls_copies[k];
                owned += bs.cls_owned[k];
            }
        const double bytes = (double)copies * (16.0 * sizeof(TC) + 8.0 + 2.0 * sizeof(T)) + 8.0 * (double)owned;
#define DM_SCHWARZ(RV, NV)                                                                                         \
    if (bs.fixed)                                                                                                  \
        launch_b(name, bytes, k_band_schwarz<T, TC, RV, NV, true>, count, NV, smem, s, first, bs.off, bs.copy,     \
                 bs.pos, bs.dims, bs.org, bs.vals, bs.ncopies, band, invD, f, (const T*)x, u, omega, sweeps, g,    \
                 bs.maxbox, bs.maxrows);                                                                         \
    else                                                                                                           \
    launch_b(name, bytes, k_band_schwarz<T, TC, RV, NV, false>, count, NV, smem, s, first, bs.off, bs.copy,      \
             bs.pos, bs.dims, bs.org, bs.vals, bs.ncopies, band, invD, f, (const T*)x, u, omega, sweeps, g,       \
             bs.maxbox, bs.maxrows)
        if (nt == 256) DM_SCHWARZ(1, 256);
        else if (R == 1) DM_SCHWARZ(1, 512);
        else if (R == 2) DM_SCHWARZ(2, 512);
        else if (R == 4) DM_SCHWARZ(4, 512);
        else DM_SCHWARZ(0, 512);
#undef DM_SCHWARZ
    }
    if (forked)
        for (int a = 0; a < std::min(nl - 1, fk->naux); ++a) {
            DM_CUDA(cudaEventRecord(fk->join[a], fk->aux[a]));
            DM_CUDA(cudaStreamWaitEvent(s0, fk->join[a], 0));
        }
    launch_b(stencil_name("band_add", prec_index<T>(), ST_JACOBI, fine), (double)nband * (12.0 + 2.0 * sizeof(T)),
             k_band_add<T>, (nband + 255) / 256, 256, 0, s0, band, nband, (const double*)u, x);
}

// Allow each variant the device's opt-in shared memory less its static share;
// the largest subdomain box must fit in it.
template <typename K>
void allow_smem(K kernel, size_t need) {
    int dev = 0, optin = 0;
    DM_CUDA(cudaGetDevice(&dev));
    DM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    DM_CUDA(cudaFuncGetAttributes(&fa, kernel));
    const long long limit = (long long)optin - (long long)fa.sharedSizeBytes;
    DM_REQUIRE((long long)need <= limit, DM_ERR_INVALID_ARG,
               "band brick too large: a subdomain's local box exceeds shared memory (use a smaller brick)");
    DM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit));
}

template <typename T, typename TC>
void band_schwarz_prepare(const SchwarzLayout& sl) {
    for (int cl = 0; cl < kSchwarzClasses; ++cl) {
        if (sl.cls_count[cl] == 0) continue;
        int R, nt;
        class_shape<T>(cl, R, nt);
        const size_t need = schwarz_smem<T>(sl.maxbox, sl.maxrows, R);
        const bool fx = sl.fixed;
        if (nt == 256) fx ? allow_smem(k_band_schwarz<T, TC, 1, 256, true>, need)
                          : allow_smem(k_band_schwarz<T, TC, 1, 256, false>, need);
        else if (R == 1) fx ? allow_smem(k_band_schwarz<T, TC, 1, 512, true>, need)
                            : allow_smem(k_band_schwarz<T, TC, 1, 512, false>, need);
        else if (R == 2) fx ? allow_smem(k_band_schwarz<T, TC, 2, 512, true>, need)
                            : allow_smem(k_band_schwarz<T, TC, 2, 512, false>, need);
        else if (R == 4) fx ? allow_smem(k_band_schwarz<T, TC, 4, 512, true>, need)
                            : allow_smem(k_band_schwarz<T, TC, 4, 512, false>, need);
        else fx ? allow_smem(k_band_schwarz<T, TC, 0, 512, true>, need)
                : allow_smem(k_band_schwarz<T, TC, 0, 512, false>, need);
    }
}

#define DM_INST(T, TC)                                                                                           \
    template void band_schwarz<T, TC>(const BandSchwarz<TC>&, const TC*, const Grid3&, const int*, int, const T*, \
                                      T*, double*, double, int, bool, cudaStream_t, const Fork*);                \
    template void band_schwarz_prepare<T, TC>(const SchwarzLayout&);
DM_INST(double, double)
DM_INST(float, float)
DM_INST(__nv_bfloat16, float)
#undef DM_INST

}  // namespace dm
