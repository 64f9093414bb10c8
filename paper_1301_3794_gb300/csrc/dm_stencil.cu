// Matrix-free Dey--Mittra operators on the padded node grid.
//
// Vector operator (Eq. discLaplDM):  y = (K - sigma A) b,
//     K = C L C^T + A D^T V^-1 D A
// with, per face, the Faraday loop of Eq. farInt weighted by the edge
// fractions L, and the grad-div term built from the Dey--Mittra divergence
// V^-1 D A of Eq. divBDM (Gauss's law on the uncovered cell volume, Eq.
// divBInt).  The curl of b on an edge, (C^T b):
//     x-edge: (b_y(k-1) - b_y(k))/dz + (b_z(k) - b_z(j-1))/dy
//     y-edge: (b_x(k) - b_x(k-1))/dz + (b_z(i-1) - b_z(i))/dx
//     z-edge: (b_x(j-1) - b_x(j))/dy + (b_y(i) - b_y(i-1))/dx
// and of the edge field e on a face, (C e):
//     x-face: (e_z(j+1) - e_z(j))/dy - (e_y(k+1) - e_y(k))/dz   (and cyclic).
// The divergence psi = V^-1 sum_faces +-A b / h (Eq. divBInt) and the
// gradient (D^T psi)_x(i) = (psi(i-1) - psi(i))/dx (Eq. gradPhi, sign of -grad).
//
// Scalar operator inside the projection (Eq. proj): S = D A D^T on cells.
#include "dm_common.cuh"
#include "dm_ff.cuh"

#include <atomic>
#include <mutex>
#include <set>

namespace dm {

namespace {

constexpr int BX = 32, BY = 4, BZ = 2;
const dim3 kBlock(BX, BY, BZ);
inline dim3 node_grid(const Grid3& g, int extra = 1) {
    return dim3((g.nx + extra + BX - 1) / BX, (g.ny + extra + BY - 1) / BY, (g.nz + extra + BZ - 1) / BZ);
}

// Field accessor over a padded 3-component vector in storage type T.
template <typename T, typename C>
struct VecAcc {
    const T* __restrict__ x;
    int np;
    __device__ __forceinline__ C operator()(int c, int p) const { return (C)to_c(x[c * np + p]); }
};
// Accessor of the first damped Jacobi iterate from zero, omega invD f, rounded
// to the storage type exactly as k_jacobi_zero stores it: the JACOBI2Z stencil
// reads its x through this instead of from a vector that pass would write.
template <typename T, typename TC, typename C>
struct Jac0Acc {
    const T* __restrict__ f;
    const TC* __restrict__ invD;
    C om;
    int np;
    __device__ __forceinline__ C operator()(int c, int p) const {
        const int q = c * np + p;
        return (C)to_c(to_store<T>(om * (C)invD[q] * (C)to_c(f[q])));
    }
};
template <typename T, typename TC, typename C, int MODE>
__device__ __forceinline__ auto x_acc(const T* x, const T* f, const TC* invD, C om, int np) {
    if constexpr (MODE == ST_JACOBI2Z)
        return Jac0Acc<T, TC, C>{f, invD, om, np};
    else
        return VecAcc<T, C>{x, np};
}
// Accessor of the unit vector e_q (packed index q = c*np + p); used to build
// the coarsest matrix column by column from the same stencil.
template <typename C>
struct UnitAcc {
    int q, np;
    __device__ __forceinline__ C operator()(int c, int p) const { return (c * np + p == q) ? C(1) : C(0); }
};

template <typename C, typename TC>
struct Coef {
    const TC* __restrict__ A;
    const TC* __restrict__ L;
    const TC* __restrict__ invV;
    int np;
    __device__ __forceinline__ C a(int c, int p) const { return (C)A[c * np + p]; }
    __device__ __forceinline__ C l(int c, int p) const { return (C)L[c * np + p]; }
    __device__ __forceinline__ C iv(int p) const { return (C)invV[p]; }
};

// L-weighted curl of b on the edges of component 0/1/2 at node p
template <typename C, typename TC, typename Acc>
__device__ __forceinline__ C edge_x(const Coef<C, TC>& cf, const Acc& b, int p, int Y, int Z, C rdy, C rdz) {
    return cf.l(0, p) * ((b(1, p - Z) - b(1, p)) * rdz + (b(2, p) - b(2, p - Y)) * rdy);
}
template <typename C, typename TC, typename Acc>
__device__ __forceinline__ C edge_y(const Coef<C, TC>& cf, const Acc& b, int p, int X, int Z, C rdx, C rdz) {
    return cf.l(1, p) * ((b(0, p) - b(0, p - Z)) * rdz + (b(2, p - X) - b(2, p)) * rdx);
}
template <typename C, typename TC, typename Acc>
__device__ __forceinline__ C edge_z(const Coef<C, TC>& cf, const Acc& b, int p, int X, int Y, C rdx, C rdy) {
    return cf.l(2, p) * ((b(0, p - Y) - b(0, p)) * rdy + (b(1, p) - b(1, p - X)) * rdx);
}
// Dey--Mittra divergence of cell p: V^-1 (sum of outward A b / h)
template <typename C, typename TC, typename Acc>
__device__ __forceinline__ C cell_psi(const Coef<C, TC>& cf, const Acc& b, int p, int X, int Y, int Z, C rdx, C rdy,
                                      C rdz) {
    const C fx = cf.a(0, p + X) * b(0, p + X) - cf.a(0, p) * b(0, p);
    const C fy = cf.a(1, p + Y) * b(1, p + Y) - cf.a(1, p) * b(1, p);
    const C fz = cf.a(2, p + Z) * b(2, p + Z) - cf.a(2, p) * b(2, p);
    return cf.iv(p) * (fx * rdx + fy * rdy + fz * rdz);
}

// (K - sigma A) b at the three faces of node p
template <typename C, typename TC, typename Acc>
__device__ __forceinline__ void node_K(const Coef<C, TC>& cf, const Acc& b, int p, int X, int Y, int Z, C rdx, C rdy,
                                       C rdz, C sigma, C out[3]) {
    const C ex0 = edge_x(cf, b, p, Y, Z, rdy, rdz);
    const C exZ = edge_x(cf, b, p + Z, Y, Z, rdy, rdz);
    const C exY = edge_x(cf, b, p + Y, Y, Z, rdy, rdz);
    const C ey0 = edge_y(cf, b, p, X, Z, rdx, rdz);
    const C eyZ = edge_y(cf, b, p + Z, X, Z, rdx, rdz);
    const C eyX = edge_y(cf, b, p + X, X, Z, rdx, rdz);
    const C ez0 = edge_z(cf, b, p, X, Y, rdx, rdy);
    const C ezY = edge_z(cf, b, p + Y, X, Y, rdx, rdy);
    const C ezX = edge_z(cf, b, p + X, X, Y, rdx, rdy);
    const C ps0 = cell_psi(cf, b, p, X, Y, Z, rdx, rdy, rdz);
    const C psX = cell_psi(cf, b, p - X, X, Y, Z, rdx, rdy, rdz);
    const C psY = cell_psi(cf, b, p - Y, X, Y, Z, rdx, rdy, rdz);
    const C psZ = cell_psi(cf, b, p - Z, X, Y, Z, rdx, rdy, rdz);
    const C ax = cf.a(0, p), ay = cf.a(1, p), az = cf.a(2, p);
    const C yx = (ezY - ez0) * rdy - (eyZ - ey0) * rdz + ax * ((psX - ps0) * rdx - sigma * b(0, p));
    const C yy = (exZ - ex0) * rdz - (ezX - ez0) * rdx + ay * ((psY - ps0) * rdy - sigma * b(1, p));
    const C yz = (eyX - ey0) * rdx - (exY - ex0) * rdy + az * ((psZ - ps0) * rdz - sigma * b(2, p));
    out[0] = ax > C(0) ? yx : C(0);
    out[1] = ay > C(0) ? yy : C(0);
    out[2] = az > C(0) ? yz : C(0);
}

// (K - sigma A) b at one face (component c, node p)
template <typename C, typename TC, typename Acc>
__device__ __forceinline__ C face_K(const Coef<C, TC>& cf, const Acc& b, int c, int p, int X, int Y, int Z, C rdx,
                                    C rdy, C rdz, C sigma) {
    const C a = cf.a(c, p);
    if (!(a > C(0))) return C(0);
    const C ps0 = cell_psi(cf, b, p, X, Y, Z, rdx, rdy, rdz);
    if (c == 0) {
        const C ez0 = edge_z(cf, b, p, X, Y, rdx, rdy), ezY = edge_z(cf, b, p + Y, X, Y, rdx, rdy);
        const C ey0 = edge_y(cf, b, p, X, Z, rdx, rdz), eyZ = edge_y(cf, b, p + Z, X, Z, rdx, rdz);
        const C psm = cell_psi(cf, b, p - X, X, Y, Z, rdx, rdy, rdz);
        return (ezY - ez0) * rdy - (eyZ - ey0) * rdz + a * ((psm - ps0) * rdx - sigma * b(0, p));
    } else if (c == 1) {
        const C ex0 = edge_x(cf, b, p, Y, Z, rdy, rdz), exZ = edge_x(cf, b, p + Z, Y, Z, rdy, rdz);
        const C ez0 = edge_z(cf, b, p, X, Y, rdx, rdy), ezX = edge_z(cf, b, p + X, X, Y, rdx, rdy);
        const C psm = cell_psi(cf, b, p - Y, X, Y, Z, rdx, rdy, rdz);
        return (exZ - ex0) * rdz - (ezX - ez0) * rdx + a * ((psm - ps0) * rdy - sigma * b(1, p));
    } else {
        const C ey0 = edge_y(cf, b, p, X, Z, rdx, rdz), eyX = edge_y(cf, b, p + X, X, Z, rdx, rdz);
        const C ex0 = edge_x(cf, b, p, Y, Z, rdy, rdz), exY = edge_x(cf, b, p + Y, Y, Z, rdy, rdz);
        const C psm = cell_psi(cf, b, p - Z, X, Y, Z, rdx, rdy, rdz);
        return (eyX - ey0) * rdx - (exY - ex0) * rdy + a * ((psm - ps0) * rdz - sigma * b(2, p));
    }
}

template <typename T, typename TC, int MODE>
__global__ void k_vec_stencil(Grid3 g, const TC* __restrict__ A, const TC* __restrict__ L,
                              const TC* __restrict__ invV, const TC* __restrict__ invD,
                              typename Compute<T>::type sigma, const T* __restrict__ x, const T* __restrict__ f,
                              T* __restrict__ y, typename Compute<T>::type omega, const int* __restrict__ tiles) {
    using C = typename Compute<T>::type;
    int i, j, k;
    block_node(g, tiles, i, j, k);
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int p = g.idx(i, j, k);
    const int N = g.np;
    Coef<C, TC> cf{A, L, invV, N};
    const auto b = x_acc<T, TC, C, MODE>(x, f, invD, omega, N);
    C out[3];
    node_K(cf, b, p, 1, g.sx, g.sxy, inv_h<C>(g, 0), inv_h<C>(g, 1), inv_h<C>(g, 2), sigma, out);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int q = c * N + p;
        C v = out[c];
        if (MODE == ST_RESID) {
            v = (C)to_c(f[q]) - v;
        } else if (MODE == ST_JACOBI) {
            v = (C)to_c(x[q]) + omega * (C)invD[q] * ((C)to_c(f[q]) - v);
        } else if (MODE == ST_JACOBI2Z) {
            v = b(c, p) + omega * (C)invD[q] * ((C)to_c(f[q]) - v);
        }
        y[q] = to_store<T>(v);
    }
}

// Tiled form of k_vec_stencil: one active tile of TX x SY x SZ nodes per
// block.  The L-weighted edge curls and cell divergences the tile's faces need
// are computed once into shared memory (ex, ey, ez on the tile plus one layer
// above, psi on the tile plus one layer below), then every thread forms its
// node's three face outputs from them.  Same arithmetic as node_K.  The tile
// shape (SY, SZ) is chosen per level by the autotuner.
template <typename T, typename TC, int MODE, int SY, int SZ>
__global__ void __launch_bounds__(TX * SY * SZ) k_vec_stencil_tiled(
    Grid3 g, const TC* __restrict__ A, const TC* __restrict__ L, const TC* __restrict__ invV,
    const TC* __restrict__ invD, typename Compute<T>::type sigma, const T* __restrict__ x, const T* __restrict__ f,
    T* __restrict__ y, typename Compute<T>::type omega, const int* __restrict__ tiles) {
    using C = typename Compute<T>::type;
    constexpr int PSI_X = TX + 1, PSI_Y = SY + 1, PSI_Z = SZ + 1;   // psi: i0-1 .. i0+TX-1 (and j, k alike)
    constexpr int EX_X = TX, EX_Y = SY + 1, EX_Z = SZ + 1;          // ex:  i0 .. i0+TX-1, j0 .. j0+SY, k0 .. k0+SZ
    constexpr int EY_X = TX + 1, EY_Y = SY, EY_Z = SZ + 1;
    constexpr int EZ_X = TX + 1, EZ_Y = SY + 1, EZ_Z = SZ;
    constexpr int N_PSI = PSI_X * PSI_Y * PSI_Z, N_EX = EX_X * EX_Y * EX_Z, N_EY = EY_X * EY_Y * EY_Z,
                  N_EZ = EZ_X * EZ_Y * EZ_Z;
    constexpr int NT = TX * SY * SZ;
    __shared__ C s_psi[N_PSI], s_ex[N_EX], s_ey[N_EY], s_ez[N_EZ];
    const int t = tiles[blockIdx.x];
    const int nti = (g.nx + TX) / TX, ntj = (g.ny + SY) / SY;
    const int i0 = (t % nti) * TX, j0 = ((t / nti) % ntj) * SY, k0 = (t / (nti * ntj)) * SZ;
    const int X = 1, Y = g.sx, Z = g.sxy, N = g.np;
    const C rdx = inv_h<C>(g, 0), rdy = inv_h<C>(g, 1), rdz = inv_h<C>(g, 2);
    Coef<C, TC> cf{A, L, invV, N};
    const auto b = x_acc<T, TC, C, MODE>(x, f, invD, omega, N);
    const int tid = threadIdx.x + TX * (threadIdx.y + SY * threadIdx.z);
    for (int e = tid; e < N_PSI; e += NT) {
        const int li = e % PSI_X, lj = (e / PSI_X) % PSI_Y, lk = e / (PSI_X * PSI_Y);
        const int i = i0 - 1 + li, j = j0 - 1 + lj, k = k0 - 1 + lk;
        C v = C(0);
        if (i >= 0 && j >= 0 && k >= 0 && i < g.nx && j < g.ny && k < g.nz)
            v = cell_psi(cf, b, g.idx(i, j, k), X, Y, Z, rdx, rdy, rdz);
        s_psi[e] = v;
    }
    for (int e = tid; e < N_EX; e += NT) {
        const int li = e % EX_X, lj = (e / EX_X) % EX_Y, lk = e / (EX_X * EX_Y);
        const int i = i0 + li, j = j0 + lj, k = k0 + lk;
        C v = C(0);
        if (i < g.nx && j <= g.ny && k <= g.nz) v = edge_x(cf, b, g.idx(i, j, k), Y, Z, rdy, rdz);
        s_ex[e] = v;
    }
    for (int e = tid; e < N_EY; e += NT) {
        const int li = e % EY_X, lj = (e / EY_X) % EY_Y, lk = e / (EY_X * EY_Y);
        const int i = i0 + li, j = j0 + lj, k = k0 + lk;
        C v = C(0);
        if (i <= g.nx && j < g.ny && k <= g.nz) v = edge_y(cf, b, g.idx(i, j, k), X, Z, rdx, rdz);
        s_ey[e] = v;
    }
    for (int e = tid; e < N_EZ; e += NT) {
        const int li = e % EZ_X, lj = (e / EZ_X) % EZ_Y, lk = e / (EZ_X * EZ_Y);
        const int i = i0 + li, j = j0 + lj, k = k0 + lk;
        C v = C(0);
        if (i <= g.nx && j <= g.ny && k < g.nz) v = edge_z(cf, b, g.idx(i, j, k), X, Y, rdx, rdy);
        s_ez[e] = v;
    }
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int i = i0 + tx, j = j0 + ty, k = k0 + tz;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int p = g.idx(i, j, k);
    auto PSI = [&](int a, int b_, int c) { return s_psi[(c * PSI_Y + b_) * PSI_X + a]; };
    auto EXS = [&](int a, int b_, int c) { return s_ex[(c * EX_Y + b_) * EX_X + a]; };
    auto EYS = [&](int a, int b_, int c) { return s_ey[(c * EY_Y + b_) * EY_X + a]; };
    auto EZS = [&](int a, int b_, int c) { return s_ez[(c * EZ_Y + b_) * EZ_X + a]; };
    const C ps0 = PSI(tx + 1, ty + 1, tz + 1);
    const C ax = cf.a(0, p), ay = cf.a(1, p), az = cf.a(2, p);
    C out[3];
    out[0] = (EZS(tx, ty + 1, tz) - EZS(tx, ty, tz)) * rdy - (EYS(tx, ty, tz + 1) - EYS(tx, ty, tz)) * rdz +
             ax * ((PSI(tx, ty + 1, tz + 1) - ps0) * rdx - sigma * b(0, p));
    out[1] = (EXS(tx, ty, tz + 1) - EXS(tx, ty, tz)) * rdz - (EZS(tx + 1, ty, tz) - EZS(tx, ty, tz)) * rdx +
             ay * ((PSI(tx + 1, ty, tz + 1) - ps0) * rdy - sigma * b(1, p));
    out[2] = (EYS(tx + 1, ty, tz) - EYS(tx, ty, tz)) * rdx - (EXS(tx, ty + 1, tz) - EXS(tx, ty, tz)) * rdy +
             az * ((PSI(tx + 1, ty + 1, tz) - ps0) * rdz - sigma * b(2, p));
    const C av[3] = {ax, ay, az};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int q = c * N + p;
        C v = av[c] > C(0) ? out[c] : C(0);
        if (MODE == ST_RESID) {
            v = (C)to_c(f[q]) - v;
        } else if (MODE == ST_JACOBI) {
            v = (C)to_c(x[q]) + omega * (C)invD[q] * ((C)to_c(f[q]) - v);
        } else if (MODE == ST_JACOBI2Z) {
            v = b(c, p) + omega * (C)invD[q] * ((C)to_c(f[q]) - v);
        }
        y[q] = to_store<T>(v);
    }
}

// z-marching form of the same operator: a block of TX x SY threads owns a
// TX x SY column of nodes and walks up to KZ planes along z.  Two planes of the
// inputs (b and A, each with a one-node ring around the column) are staged in
// shared memory; for each plane the block forms the cell divergences and z-edge
// curls of that plane and the x/y-edge curls of the plane above (kept for two
// planes), then every thread forms its node's three face outputs.  Each thread
// loads and computes the entries of its own node, and the ring and the one-node
// borders of the divergence and curl tiles are spread one entry per thread over
// the block, so index arithmetic is done once per block rather than per entry.
// Every input value is read from global memory about once per block (the ring
// and the one plane below and above the column are the only re-reads), and each
// curl and divergence is computed once.  The global loads of the next plane are
// issued into registers before the current plane's outputs are formed, so their
// latency overlaps that work.  Entries outside [-1, n+1] along x or y are taken
// as zero; inside that box the padded layout already holds zeros at every
// position that is not an element of the grid.
template <typename T, typename TC, int MODE, int SY, int KZ>
__global__ void __launch_bounds__(TX * SY, (std::is_same<T, double>::value ? 512 : 768) / (TX * SY)) k_vec_stencil_march(
    Grid3 g, const TC* __restrict__ A, const TC* __restrict__ L, const TC* __restrict__ invV,
    const TC* __restrict__ invD, typename Compute<T>::type sigma, const T* __restrict__ x, const T* __restrict__ f,
    T* __restrict__ y, typename Compute<T>::type omega, const int* __restrict__ tiles) {
    using C = typename Compute<T>::type;
    constexpr int RW = TX + 2, RH = SY + 2, RP = RW * RH;   // ring plane: i0-1 .. i0+TX, j0-1 .. j0+SY
    constexpr int NT = TX * SY;
    constexpr int W1 = TX + 1;
    constexpr int NRH = 2 * TX + 2 * RH;   // ring border entries
    constexpr int NPH = W1 + SY;           // psi border: row j0-1 (i0-1 .. i0+TX-1), column i0-1 (j0 .. j0+SY-1)
    constexpr int NZH = W1 + SY;           // z-edge border: row j0+SY (i0 .. i0+TX), column i0+TX (j0 .. j0+SY-1)
    constexpr int NXH = TX;                // x-edge border: row j0+SY (i0 .. i0+TX-1)
    constexpr int NYH = SY;                // y-edge border: column i0+TX (j0 .. j0+SY-1)
    static_assert(NRH <= NT && NPH + NZH + NXH + NYH <= NT, "one border entry per thread");
    __shared__ C s_ring[2][6 * RP];        // b_x, b_y, b_z, A_x, A_y, A_z (blocks of RP) of two planes
    __shared__ C s_ex[2][(SY + 1) * TX];   // x-edges i0 .. i0+TX-1, j0 .. j0+SY (two planes)
    __shared__ C s_ey[2][SY * W1];         // y-edges i0 .. i0+TX,   j0 .. j0+SY-1 (two planes)
    __shared__ C s_ez[(SY + 1) * W1];      // z-edges i0 .. i0+TX,   j0 .. j0+SY
    __shared__ C s_psi[(SY + 1) * W1];     // cells   i0-1 .. i0+TX-1, j0-1 .. j0+SY-1
    const int t = tiles[blockIdx.x];
    const int nti = (g.nx + TX) / TX, ntj = (g.ny + SY) / SY;
    const int i0 = (t % nti) * TX, j0 = ((t / nti) % ntj) * SY, k0 = (t / (nti * ntj)) * KZ;
    const int kend = min(k0 + KZ - 1, g.nz);
    const int N = g.np, Z = g.sxy;
    const int ilim = g.nx + 1, jlim = g.ny + 1;
    const C rdx = inv_h<C>(g, 0), rdy = inv_h<C>(g, 1), rdz = inv_h<C>(g, 2);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + TX * ty;
    // this thread's node
    const int i = i0 + tx, j = j0 + ty;
    const bool inb = i <= ilim && j <= jlim;          // inside the padded box
    const bool own = i <= g.nx && j <= g.ny;          // an output node
    const int p0 = g.idx(i, j, 0);
    const int rown = (ty + 1) * RW + tx + 1;          // ring position of the node
    // ring border entry of this thread
    int hli = 0, hlj = 0;
    if (tid < TX) { hli = tid + 1; hlj = 0; }
    else if (tid < 2 * TX) { hli = tid - TX + 1; hlj = RH - 1; }
    else if (tid < 2 * TX + RH) { hli = 0; hlj = tid - 2 * TX; }
    else { hli = RW - 1; hlj = tid - 2 * TX - RH; }
    const bool hval = tid < NRH && i0 - 1 + hli <= ilim && j0 - 1 + hlj <= jlim;
    const int hp0 = hval ? g.idx(i0 - 1 + hli, j0 - 1 + hlj, 0) : 0;
    const int rh = hlj * RW + hli;
    // border entry of the divergence / curl tiles: role 0 psi, 1 z-edge, 2 x-edge, 3 y-edge, -1 none
    int role = -1, di = 0, dj = 0, dsm = 0;
    if (tid < NPH) {
        role = 0;
        if (tid < W1) { di = i0 - 1 + tid; dj = j0 - 1; dsm = tid; }
        else { di = i0 - 1; dj = j0 + (tid - W1); dsm = (tid - W1 + 1) * W1; }
    } else if (tid < NPH + NZH) {
        const int e = tid - NPH;
        role = 1;
        if (e < W1) { di = i0 + e; dj = j0 + SY; dsm = SY * W1 + e; }
        else { di = i0 + TX; dj = j0 + (e - W1); dsm = (e - W1) * W1 + TX; }
    } else if (tid < NPH + NZH + NXH) {
        const int e = tid - NPH - NZH;
        role = 2; di = i0 + e; dj = j0 + SY; dsm = SY * TX + e;
    } else if (tid < NPH + NZH + NXH + NYH) {
        const int e = tid - NPH - NZH - NXH;
        role = 3; di = i0 + TX; dj = j0 + e; dsm = e * W1 + TX;
    }
    const bool dval = role >= 0 && di <= ilim && dj <= jlim;
    const int dp0 = dval ? g.idx(di, dj, 0) : 0;
    // ring entry of array a (0..2: b, 3..5: A) at node (ii, jj) of the plane in `slot`
    auto R = [&](int slot, int a, int ii, int jj) -> C { return s_ring[slot][a * RP + (jj - j0 + 1) * RW + (ii - i0 + 1)]; };
    const auto xa = x_acc<T, TC, C, MODE>(x, f, invD, omega, N);
    // prefetch registers: ring entries of the node and of the border entry, coefficients, f and 1/D
    C pn[6], ph[6], cv = C(0), cz = C(0), cx = C(0), cy = C(0), hc = C(0), he = C(0), pf[3], pd[3];
    auto fetch_ring = [&](int k) {
        const int pn_ = p0 + k * Z, ph_ = hp0 + k * Z;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pn[c] = inb ? xa(c, pn_) : C(0);
            pn[3 + c] = inb ? (C)A[c * N + pn_] : C(0);
            ph[c] = hval ? xa(c, ph_) : C(0);
            ph[3 + c] = hval ? (C)A[c * N + ph_] : C(0);
        }
    };
    auto store_ring = [&](int slot) {
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            s_ring[slot][a * RP + rown] = pn[a];
            if (tid < NRH) s_ring[slot][a * RP + rh] = ph[a];
        }
    };
    // 1/V and L_z at plane k: the node's, and the border entry's for roles 0 and 1
    auto fetch_cells = [&](int k) {
        cv = inb ? (C)invV[p0 + k * Z] : C(0);
        cz = inb ? (C)L[2 * N + p0 + k * Z] : C(0);
        hc = C(0);
        if (dval && role == 0) hc = (C)invV[dp0 + k * Z];
        if (dval && role == 1) hc = (C)L[2 * N + dp0 + k * Z];
    };
    // L_x and L_y at plane kp: the node's, and the border entry's for roles 2 and 3
    auto fetch_edges = [&](int kp) {
        cx = inb ? (C)L[p0 + kp * Z] : C(0);
        cy = inb ? (C)L[N + p0 + kp * Z] : C(0);
        he = C(0);
        if (dval && role == 2) he = (C)L[dp0 + kp * Z];
        if (dval && role == 3) he = (C)L[N + dp0 + kp * Z];
    };
    auto fetch_out = [&](int k) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pf[c] = C(0);
            pd[c] = C(0);
            if (MODE != ST_APPLY && own) {
                pf[c] = (C)to_c(f[c * N + p0 + k * Z]);
                if (MODE == ST_JACOBI || MODE == ST_JACOBI2Z) pd[c] = (C)invD[c * N + p0 + k * Z];
            }
        }
    };
    // L-weighted curls and the Dey--Mittra divergence at (ii, jj) from the ring
    auto ex_at = [&](int ii, int jj, int sm, int sp, C lx) -> C {
        return lx * ((R(sm, 1, ii, jj) - R(sp, 1, ii, jj)) * rdz + (R(sp, 2, ii, jj) - R(sp, 2, ii, jj - 1)) * rdy);
    };
    auto ey_at = [&](int ii, int jj, int sm, int sp, C ly) -> C {
        return ly * ((R(sp, 0, ii, jj) - R(sm, 0, ii, jj)) * rdz + (R(sp, 2, ii - 1, jj) - R(sp, 2, ii, jj)) * rdx);
    };
    auto ez_at = [&](int ii, int jj, int s0, C lz) -> C {
        return lz * ((R(s0, 0, ii, jj - 1) - R(s0, 0, ii, jj)) * rdy + (R(s0, 1, ii, jj) - R(s0, 1, ii - 1, jj)) * rdx);
    };
    auto psi_at = [&](int ii, int jj, int s0, int s1, C iv) -> C {
        const C fx = R(s0, 3, ii + 1, jj) * R(s0, 0, ii + 1, jj) - R(s0, 3, ii, jj) * R(s0, 0, ii, jj);
        const C fy = R(s0, 4, ii, jj + 1) * R(s0, 1, ii, jj + 1) - R(s0, 4, ii, jj) * R(s0, 1, ii, jj);
        const C fz = R(s1, 5, ii, jj) * R(s1, 2, ii, jj) - R(s0, 5, ii, jj) * R(s0, 2, ii, jj);
        return iv * (fx * rdx + fy * rdy + fz * rdz);
    };
    // x- and y-edge curls of plane kp (ring slots: sm = plane kp-1, sp = plane kp) into edge slot es
    auto edges_xy = [&](int sm, int sp, int es) {
        s_ex[es][ty * TX + tx] = inb ? ex_at(i, j, sm, sp, cx) : C(0);
        s_ey[es][ty * W1 + tx] = inb ? ey_at(i, j, sm, sp, cy) : C(0);
        if (role == 2) s_ex[es][dsm] = dval ? ex_at(di, dj, sm, sp, he) : C(0);
        if (role == 3) s_ey[es][dsm] = dval ? ey_at(di, dj, sm, sp, he) : C(0);
    };
    // cell divergences and z-edge curls of plane k (ring slots: s0 = plane k, s1 = plane k+1)
    auto psi_ez = [&](int s0, int s1) {
        s_psi[(ty + 1) * W1 + tx + 1] = inb ? psi_at(i, j, s0, s1, cv) : C(0);
        s_ez[ty * W1 + tx] = inb ? ez_at(i, j, s0, cz) : C(0);
        if (role == 0) s_psi[dsm] = dval ? psi_at(di, dj, s0, s1, hc) : C(0);
        if (role == 1) s_ez[dsm] = dval ? ez_at(di, dj, s0, hc) : C(0);
    };
    // prologue: planes k0-1 (ring slot 0) and k0 (slot 1); edges of plane k0 (edge slot 0);
    // psi(k0-1) at this thread's node; then the loads of the first iteration
    fetch_ring(k0 - 1);
    store_ring(0);
    fetch_ring(k0);
    store_ring(1);
    fetch_edges(k0);
    __syncthreads();
    edges_xy(0, 1, 0);
    C psi_below = own ? psi_at(i, j, 0, 1, (C)invV[p0 + (k0 - 1) * Z]) : C(0);
    fetch_ring(k0 + 1);
    fetch_cells(k0);
    fetch_edges(k0 + 1);
    for (int k = k0; k <= kend; ++k) {
        const int s0 = (k - k0 + 1) & 1, s1 = s0 ^ 1;   // ring slots of planes k and k+1
        const int e0 = (k - k0) & 1, e1 = e0 ^ 1;        // edge slots of planes k and k+1
        fetch_out(k);     // f and 1/D of this plane: in flight through the barriers below
        __syncthreads();
        store_ring(s1);
        __syncthreads();
        psi_ez(s0, s1);
        edges_xy(s0, s1, e1);
        if (k < kend) {   // loads of the next iteration, in flight while this plane's outputs are formed
            fetch_ring(k + 2);
            fetch_cells(k + 1);
            fetch_edges(k + 2);
        }
        __syncthreads();
        if (own) {
            const C ps0 = s_psi[(ty + 1) * W1 + tx + 1];
            const C ez0 = s_ez[ty * W1 + tx];
            const C ax = s_ring[s0][3 * RP + rown], ay = s_ring[s0][4 * RP + rown], az = s_ring[s0][5 * RP + rown];
            const C bx = s_ring[s0][rown], by = s_ring[s0][RP + rown], bz = s_ring[s0][2 * RP + rown];
            C out[3];
            out[0] = (s_ez[(ty + 1) * W1 + tx] - ez0) * rdy - (s_ey[e1][ty * W1 + tx] - s_ey[e0][ty * W1 + tx]) * rdz +
                     ax * ((s_psi[(ty + 1) * W1 + tx] - ps0) * rdx - sigma * bx);
            out[1] = (s_ex[e1][ty * TX + tx] - s_ex[e0][ty * TX + tx]) * rdz - (s_ez[ty * W1 + tx + 1] - ez0) * rdx +
                     ay * ((s_psi[ty * W1 + tx + 1] - ps0) * rdy - sigma * by);
            out[2] = (s_ey[e0][ty * W1 + tx + 1] - s_ey[e0][ty * W1 + tx]) * rdx -
                     (s_ex[e0][(ty + 1) * TX + tx] - s_ex[e0][ty * TX + tx]) * rdy +
                     az * ((psi_below - ps0) * rdz - sigma * bz);
            const C av[3] = {ax, ay, az}, bv[3] = {bx, by, bz};
            const int p = p0 + k * Z;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                C v = av[c] > C(0) ? out[c] : C(0);
                if (MODE == ST_RESID) {
                    v = pf[c] - v;
                } else if (MODE == ST_JACOBI || MODE == ST_JACOBI2Z) {
                    v = bv[c] + omega * pd[c] * (pf[c] - v);
                }
                y[c * N + p] = to_store<T>(v);
            }
            psi_below = ps0;
        }
    }
}

template <typename T, typename TC>
__global__ void k_jacobi_zero(Domain d, const TC* __restrict__ invD, const T* __restrict__ f, T* __restrict__ y,
                              typename Compute<T>::type om) {
    using C = typename Compute<T>::type;
    for_each_entry(d, [&](long long q) { y[q] = to_store<T>(om * (C)invD[q] * (C)to_c(f[q])); });
}

// Rows of K - sigma A for the band faces in the fixed 15-slot form of
// band_slot (slot-major: slot e of band face t at [e * nband + t]); each
// coefficient is face_K of the column's unit vector, the same arithmetic as
// every other use of the operator.
__global__ void k_band_slots(Grid3 g, const double* __restrict__ A, const double* __restrict__ L,
                             const double* __restrict__ invV, double sigma, const int* __restrict__ band, int nband,
                             double* __restrict__ vals) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nband) return;
    const int q = band[t];
    const int c = q / g.np, p = q - c * g.np;
    Coef<double, double> cf{A, L, invV, g.np};
    const double rdx = g.rhx, rdy = g.rhy, rdz = g.rhz;
    for (int e = 0; e < kBandSlots; ++e) {
        UnitAcc<double> b{q + band_slot_offset(c, e, g.np, g.sx, g.sxy), g.np};
        vals[(size_t)e * nband + t] = face_K(cf, b, c, p, 1, g.sx, g.sxy, rdx, rdy, rdz, sigma);
    }
}

// diagonal of K - sigma A (x-face; other components cyclic):
//   (L_z(j) + L_z(j+1))/dy^2 + (L_y(k) + L_y(k+1))/dz^2 + A_x^2 (V^-1(i-1) + V^-1(i))/dx^2 - sigma A_x
__global__ void k_vec_diag(Grid3 g, const double* __restrict__ A, const double* __restrict__ L,
                           const double* __restrict__ invV, double sigma, double* __restrict__ d) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z * BZ + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int p = g.idx(i, j, k);
    const int X = 1, Y = g.sx, Z = g.sxy, N = g.np;
    const double rx2 = 1.0 / (g.hx * g.hx), ry2 = 1.0 / (g.hy * g.hy), rz2 = 1.0 / (g.hz * g.hz);
    const double ax = A[p], ay = A[N + p], az = A[2 * N + p];
    d[p] = ax > 0.0 ? (L[2 * N + p] + L[2 * N + p + Y]) * ry2 + (L[N + p] + L[N + p + Z]) * rz2 +
                          ax * ax * (invV[p - X] + invV[p]) * rx2 - sigma * ax
                    : 0.0;
    d[N + p] = ay > 0.0 ? (L[p] + L[p + Z]) * rz2 + (L[2 * N + p] + L[2 * N + p + X]) * rx2 +
                              ay * ay * (invV[p - Y] + invV[p]) * ry2 - sigma * ay
                        : 0.0;
    d[2 * N + p] = az > 0.0 ? (L[N + p] + L[N + p + X]) * rx2 + (L[p] + L[p + Y]) * ry2 +
                                  az * az * (invV[p - Z] + invV[p]) * rz2 - sigma * az
                            : 0.0;
}

// column `col` of the dense (K - sigma A) restricted to the listed faces
__global__ void k_vec_dense(Grid3 g, const double* __restrict__ A, const double* __restrict__ L,
                            const double* __restrict__ invV, double sigma, const int* __restrict__ list, int n,
                            double* __restrict__ M) {
    const int col = blockIdx.x;
    Coef<double, double> cf{A, L, invV, g.np};
    UnitAcc<double> b{list[col], g.np};
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const int q = list[r];
        const int c = q / g.np, p = q - c * g.np;
        M[(long long)r * n + col] = face_K(cf, b, c, p, 1, g.sx, g.sxy, g.rhx, g.rhy, g.rhz, sigma);
    }
}

// ---- scalar Laplacian S = D A D^T on cells --------------------------------------
template <typename C, typename TC, typename Acc>
__device__ __forceinline__ C cell_S(const TC* __restrict__ A, const Acc& v, int p, int X, int Y, int Z, int N, C rx2,
                                    C ry2, C rz2) {
    const C v0 = v(p);
    return ((C)A[p + X] * (v0 - v(p + X)) + (C)A[p] * (v0 - v(p - X))) * rx2 +
           ((C)A[N + p + Y] * (v0 - v(p + Y)) + (C)A[N + p] * (v0 - v(p - Y))) * ry2 +
           ((C)A[2 * N + p + Z] * (v0 - v(p + Z)) + (C)A[2 * N + p] * (v0 - v(p - Z))) * rz2;
}
template <typename T, typename C>
struct CellAcc {
    const T* __restrict__ x;
    __device__ __forceinline__ C operator()(int p) const { return (C)to_c(x[p]); }
};
template <typename C>
struct CellUnit {
    int q;
    __device__ __forceinline__ C operator()(int p) const { return p == q ? C(1) : C(0); }
};

template <typename T, typename TC, int MODE>
__global__ void k_scal_stencil(Grid3 g, const TC* __restrict__ A, const unsigned char* __restrict__ active,
                               const TC* __restrict__ invD, const T* __restrict__ x, const T* __restrict__ f,
                               T* __restrict__ y, typename Compute<T>::type omega, const int* __restrict__ tiles) {
    using C = typename Compute<T>::type;
    int i, j, k;
    block_node(g, tiles, i, j, k);
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;
    const int p = g.idx(i, j, k);
    C v = C(0);
    if (active[p]) {
        CellAcc<T, C> acc{x};
        const C rx = inv_h<C>(g, 0), ry = inv_h<C>(g, 1), rz = inv_h<C>(g, 2);
        const C sx = cell_S<C>(A, acc, p, 1, g.sx, g.sxy, g.np, rx * rx, ry * ry, rz * rz);
        if (MODE == ST_APPLY) v = sx;
        else if (MODE == ST_RESID) v = (C)to_c(f[p]) - sx;
        else v = (C)to_c(x[p]) + omega * (C)invD[p] * ((C)to_c(f[p]) - sx);
    }
    y[p] = to_store<T>(v);
}

__global__ void k_scal_diag(Grid3 g, const double* __restrict__ A, const unsigned char* __restrict__ active,
                            double* __restrict__ d) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z * BZ + threadIdx.z;
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;
    const int p = g.idx(i, j, k);
    const int X = 1, Y = g.sx, Z = g.sxy, N = g.np;
    d[p] = active[p] ? (A[p] + A[p + X]) / (g.hx * g.hx) + (A[N + p] + A[N + p + Y]) / (g.hy * g.hy) +
                           (A[2 * N + p] + A[2 * N + p + Z]) / (g.hz * g.hz)
                     : 0.0;
}

__global__ void k_scal_dense(Grid3 g, const double* __restrict__ A, const int* __restrict__ list,
                             const unsigned char* __restrict__ pinned, int n, double* __restrict__ M) {
    const int col = blockIdx.x;
    CellUnit<double> u{list[col]};
    const double rx2 = 1.0 / (g.hx * g.hx), ry2 = 1.0 / (g.hy * g.hy), rz2 = 1.0 / (g.hz * g.hz);
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        double v;
        if (pinned[r] || pinned[col]) v = (r == col) ? 1.0 : 0.0;
        else v = cell_S<double>(A, u, list[r], 1, g.sx, g.sxy, g.np, rx2, ry2, rz2);
        M[(long long)r * n + col] = v;
    }
}

// s = D (A x) on cells (Eq. divBInt without the V^-1)
__global__ void k_div_a(Grid3 g, const double* __restrict__ A, const double* __restrict__ x, double* __restrict__ s,
                        const int* __restrict__ tiles) {
    int i, j, k;
    block_node(g, tiles, i, j, k);
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;
    const int p = g.idx(i, j, k);
    const int X = 1, Y = g.sx, Z = g.sxy, N = g.np;
    s[p] = (A[p + X] * x[p + X] - A[p] * x[p]) * g.rhx + (A[N + p + Y] * x[N + p + Y] - A[N + p] * x[N + p]) * g.rhy +
           (A[2 * N + p + Z] * x[2 * N + p + Z] - A[2 * N + p] * x[2 * N + p]) * g.rhz;
}

// y = x - D^T phi on open faces, (D^T phi)_x(i) = (phi(i-1) - phi(i))/dx
__global__ void k_sub_grad(Grid3 g, const double* __restrict__ A, const double* __restrict__ x,
                           const double* __restrict__ phi, double* __restrict__ y, const int* __restrict__ tiles) {
    int i, j, k;
    block_node(g, tiles, i, j, k);
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int p = g.idx(i, j, k);
    const int X = 1, Y = g.sx, Z = g.sxy, N = g.np;
    const double ph = phi[p];
    y[p] = A[p] > 0.0 ? x[p] - (phi[p - X] - ph) * g.rhx : 0.0;
    y[N + p] = A[N + p] > 0.0 ? x[N + p] - (phi[p - Y] - ph) * g.rhy : 0.0;
    y[2 * N + p] = A[2 * N + p] > 0.0 ? x[2 * N + p] - (phi[p - Z] - ph) * g.rhz : 0.0;
}

// (K - sigma A) x in float-float on the FP32 pipes, for the shifted solves'
// Krylov vectors: x is FP64, the coefficients are float-float copies of the
// level's FP64 A, L, 1/V, and every product and sum is a float-float operation
// (about 48 significant bits).  The result goes straight into the compact
// float-float vector of the FGMRES basis: out[cmap[q]] for every open face q.
// Same tiles and the same sharing of edge curls and cell divergences through
// shared memory as k_vec_stencil_tiled (32 x 4 x 2 tiles); in addition the
// block splits the x it needs (the tile with a one-node ring) into float-float
// once, into shared memory, so that each value is converted once per block.
__global__ void __launch_bounds__(TX * TY * TZ) k_vec_apply_ff(Grid3 g, const float2* __restrict__ A,
                                                               const float2* __restrict__ L,
                                                               const float2* __restrict__ invV, ffv rdx, ffv rdy,
                                                               ffv rdz, ffv sigma, const double* __restrict__ x,
                                                               const int* __restrict__ cmap, float2* __restrict__ out,
                                                               const int* __restrict__ tiles) {
    constexpr int SY = TY, SZ = TZ;
    constexpr int BXW = TX + 2, BYW = SY + 2, BZW = SZ + 2, NB = BXW * BYW * BZW;   // x: i0-1 .. i0+TX (j, k alike)
    constexpr int PSI_X = TX + 1, PSI_Y = SY + 1, PSI_Z = SZ + 1;
    constexpr int EX_X = TX, EX_Y = SY + 1, EX_Z = SZ + 1;
    constexpr int EY_X = TX + 1, EY_Y = SY, EY_Z = SZ + 1;
    constexpr int EZ_X = TX + 1, EZ_Y = SY + 1, EZ_Z = SZ;
    constexpr int N_PSI = PSI_X * PSI_Y * PSI_Z, N_EX = EX_X * EX_Y * EX_Z, N_EY = EY_X * EY_Y * EY_Z,
                  N_EZ = EZ_X * EZ_Y * EZ_Z;
    constexpr int NT = TX * SY * SZ;
    __shared__ ffv s_b[3][NB];
    __shared__ ffv s_psi[N_PSI], s_ex[N_EX], s_ey[N_EY], s_ez[N_EZ];
    const int t = tiles[blockIdx.x];
    const int nti = (g.nx + TX) / TX, ntj = (g.ny + SY) / SY;
    const int i0 = (t % nti) * TX, j0 = ((t / nti) % ntj) * SY, k0 = (t / (nti * ntj)) * SZ;
    const int X = 1, Y = g.sx, Z = g.sxy, N = g.np;
    const int tid = threadIdx.x + TX * (threadIdx.y + SY * threadIdx.z);
    // x over the box; the padded layout holds nodes -1 .. n+1 along each axis
    // (zero where no face exists), and nodes past n+1 are taken as zero
    for (int e = tid; e < NB; e += NT) {
        const int li = e % BXW, lj = (e / BXW) % BYW, lk = e / (BXW * BYW);
        const int i = i0 - 1 + li, j = j0 - 1 + lj, k = k0 - 1 + lk;
        const bool in = i <= g.nx + 1 && j <= g.ny + 1 && k <= g.nz + 1;
        const int p = in ? g.idx(i, j, k) : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) s_b[c][e] = in ? ff_from_double(x[c * N + p]) : ff_zero();
    }
    __syncthreads();
    // b(c, li, lj, lk): box coordinates (node i0-1+li ...)
    auto b = [&](int c, int li, int lj, int lk) { return s_b[c][(lk * BYW + lj) * BXW + li]; };
    auto a = [&](int c, int p) { return ff_load(A + c * N + p); };
    auto l = [&](int c, int p) { return ff_load(L + c * N + p); };
    for (int e = tid; e < N_PSI; e += NT) {
        const int li = e % PSI_X, lj = (e / PSI_X) % PSI_Y, lk = e / (PSI_X * PSI_Y);   // box coords of the cell
        const int i = i0 - 1 + li, j = j0 - 1 + lj, k = k0 - 1 + lk;
        ffv v = ff_zero();
        if (i >= 0 && j >= 0 && k >= 0 && i < g.nx && j < g.ny && k < g.nz) {
            const int p = g.idx(i, j, k);
            const ffv iv = ff_load(invV + p);
            if (iv.hi != 0.f) {
                const ffv fx = a(0, p + X) * b(0, li + 1, lj, lk) - a(0, p) * b(0, li, lj, lk);
                const ffv fy = a(1, p + Y) * b(1, li, lj + 1, lk) - a(1, p) * b(1, li, lj, lk);
                const ffv fz = a(2, p + Z) * b(2, li, lj, lk + 1) - a(2, p) * b(2, li, lj, lk);
                v = iv * (fx * rdx + fy * rdy + fz * rdz);
            }
        }
        s_psi[e] = v;
    }
    for (int e = tid; e < N_EX; e += NT) {
        const int li = e % EX_X, lj = (e / EX_X) % EX_Y, lk = e / (EX_X * EX_Y);
        const int i = i0 + li, j = j0 + lj, k = k0 + lk;
        ffv v = ff_zero();
        if (i < g.nx && j <= g.ny && k <= g.nz) {
            const ffv lv = l(0, g.idx(i, j, k));
            const int bi = li + 1, bj = lj + 1, bk = lk + 1;
            if (lv.hi != 0.f)
                v = lv * ((b(1, bi, bj, bk - 1) - b(1, bi, bj, bk)) * rdz + (b(2, bi, bj, bk) - b(2, bi, bj - 1, bk)) * rdy);
        }
        s_ex[e] = v;
    }
    for (int e = tid; e < N_EY; e += NT) {
        const int li = e % EY_X, lj = (e / EY_X) % EY_Y, lk = e / (EY_X * EY_Y);
        const int i = i0 + li, j = j0 + lj, k = k0 + lk;
        ffv v = ff_zero();
        if (i <= g.nx && j < g.ny && k <= g.nz) {
            const ffv lv = l(1, g.idx(i, j, k));
            const int bi = li + 1, bj = lj + 1, bk = lk + 1;
            if (lv.hi != 0.f)
                v = lv * ((b(0, bi, bj, bk) - b(0, bi, bj, bk - 1)) * rdz + (b(2, bi - 1, bj, bk) - b(2, bi, bj, bk)) * rdx);
        }
        s_ey[e] = v;
    }
    for (int e = tid; e < N_EZ; e += NT) {
        const int li = e % EZ_X, lj = (e / EZ_X) % EZ_Y, lk = e / (EZ_X * EZ_Y);
        const int i = i0 + li, j = j0 + lj, k = k0 + lk;
        ffv v = ff_zero();
        if (i <= g.nx && j <= g.ny && k < g.nz) {
            const ffv lv = l(2, g.idx(i, j, k));
            const int bi = li + 1, bj = lj + 1, bk = lk + 1;
            if (lv.hi != 0.f)
                v = lv * ((b(0, bi, bj - 1, bk) - b(0, bi, bj, bk)) * rdy + (b(1, bi, bj, bk) - b(1, bi - 1, bj, bk)) * rdx);
        }
        s_ez[e] = v;
    }
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int i = i0 + tx, j = j0 + ty, k = k0 + tz;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int p = g.idx(i, j, k);
    auto PSI = [&](int aa, int bb, int cc) { return s_psi[(cc * PSI_Y + bb) * PSI_X + aa]; };
    auto EXS = [&](int aa, int bb, int cc) { return s_ex[(cc * EX_Y + bb) * EX_X + aa]; };
    auto EYS = [&](int aa, int bb, int cc) { return s_ey[(cc * EY_Y + bb) * EY_X + aa]; };
    auto EZS = [&](int aa, int bb, int cc) { return s_ez[(cc * EZ_Y + bb) * EZ_X + aa]; };
    const ffv ps0 = PSI(tx + 1, ty + 1, tz + 1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int ci = cmap[c * N + p];
        if (ci < 0) continue;   // closed face
        const ffv av = a(c, p);
        const ffv bv = b(c, tx + 1, ty + 1, tz + 1);
        ffv v;
        if (c == 0)
            v = (EZS(tx, ty + 1, tz) - EZS(tx, ty, tz)) * rdy - (EYS(tx, ty, tz + 1) - EYS(tx, ty, tz)) * rdz +
                av * ((PSI(tx, ty + 1, tz + 1) - ps0) * rdx - sigma * bv);
        else if (c == 1)
            v = (EXS(tx, ty, tz + 1) - EXS(tx, ty, tz)) * rdz - (EZS(tx + 1, ty, tz) - EZS(tx, ty, tz)) * rdx +
                av * ((PSI(tx + 1, ty, tz + 1) - ps0) * rdy - sigma * bv);
        else
            v = (EYS(tx + 1, ty, tz) - EYS(tx, ty, tz)) * rdx - (EXS(tx, ty + 1, tz) - EXS(tx, ty, tz)) * rdy +
                av * ((PSI(tx + 1, ty + 1, tz) - ps0) * rdz - sigma * bv);
        out[ci] = make_float2(v.hi, v.lo);
    }
}

// D A D^T x on the active cells in float-float (the projection's scalar
// operator, Eq. proj), straight into the compact float-float vector of the
// scalar FGMRES basis: out[cmap[p]] for every active cell p.  x is FP64 (split
// on load), A the float-float face fractions, 1/h^2 float-float.
__global__ void k_scal_apply_ff(Grid3 g, const float2* __restrict__ A, ffv rx2, ffv ry2, ffv rz2,
                                const double* __restrict__ x, const int* __restrict__ cmap, float2* __restrict__ out,
                                const int* __restrict__ tiles) {
    int i, j, k;
    block_node(g, tiles, i, j, k);
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;
    const int p = g.idx(i, j, k);
    const int ci = cmap[p];
    if (ci < 0) return;
    const int X = 1, Y = g.sx, Z = g.sxy, N = g.np;
    auto v = [&](int q) { return ff_from_double(x[q]); };
    auto a = [&](int q) { return ff_load(A + q); };
    const ffv v0 = v(p);
    const ffv sx = (a(p + X) * (v0 - v(p + X)) + a(p) * (v0 - v(p - X))) * rx2;
    const ffv sy = (a(N + p + Y) * (v0 - v(p + Y)) + a(N + p) * (v0 - v(p - Y))) * ry2;
    const ffv sz = (a(2 * N + p + Z) * (v0 - v(p + Z)) + a(2 * N + p) * (v0 - v(p - Z))) * rz2;
    const ffv r = sx + sy + sz;
    out[ci] = make_float2(r.hi, r.lo);
}

// float-float copy of an FP64 array: hi = the double rounded to FP32, lo =
// the rest rounded (setup only, FP64 arithmetic)
__global__ void k_to_ff(long long n, const double* __restrict__ a, float2* __restrict__ out) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        const float hi = __double2float_rn(a[r]);
        out[r] = make_float2(hi, __double2float_rn(a[r] - (double)hi));
    }
}

// cmap[q] = the compact index of open face q (the position of q in the
// ascending list of open faces), -1 elsewhere
__global__ void k_compact_map(long long n3, const int* __restrict__ list, int nl, int* __restrict__ cmap) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nl; r += (long long)gridDim.x * blockDim.x)
        cmap[list[r]] = (int)r;
    (void)n3;
}

ffv host_ff(double v) {
    ffv f;
    f.hi = (float)v;
    f.lo = (float)(v - (double)f.hi);
    return f;
}

}  // namespace

void to_ff(long long n, const double* a, float2* out, cudaStream_t s) {
    launch("k_to_ff", k_to_ff, (int)std::min<long long>((n + 255) / 256, 152 * 8), 256, 0, s, n, a, out);
}

void compact_map(long long n3, const int* list, int nl, int* cmap, cudaStream_t s) {
    DM_CUDA(cudaMemsetAsync(cmap, 0xff, sizeof(int) * (size_t)n3, s));
    launch("k_compact_map", k_compact_map, (int)std::min<long long>(((long long)nl + 255) / 256, 152 * 8), 256, 0, s, n3,
           list, nl, cmap);
}

void vec_apply_ff(const Grid3& g, const int* tiles, int ntiles, const float2* A, const float2* L, const float2* invV,
                  double sigma, const double* x, const int* cmap, float2* out, cudaStream_t s) {
    if (ntiles <= 0) return;
    // bytes: per open face its x (8), A and about one L (8 each), a third of a 1/V (8), the output (8) and cmap (4)
    const double bytes = (double)g.nopen * (8.0 + 16.0 + 8.0 / 3.0 + 12.0);
    launch_b("vec_apply_ff_L0", bytes, k_vec_apply_ff, ntiles, dim3(TX, TY, TZ), 0, s, g, A, L, invV, host_ff(g.rhx),
             host_ff(g.rhy), host_ff(g.rhz), host_ff(sigma), x, cmap, out, tiles);
}

void scal_apply_ff(const Grid3& g, const int* tiles, int ntiles, const float2* A, const double* x, const int* cmap,
                   float2* out, cudaStream_t s) {
    if (ntiles <= 0) return;
    // bytes: per active cell its x (8), three float-float face fractions (24; six faces, each shared by two
    // cells), the output (8) and its compact index (4)
    const double bytes = (double)g.nact * (8.0 + 24.0 + 12.0);
    launch_b("scal_apply_ff_L0", bytes, k_scal_apply_ff, ntiles, kBlock, 0, s, g, A, host_ff(g.rhx * g.rhx),
             host_ff(g.rhy * g.rhy), host_ff(g.rhz * g.rhz), x, cmap, out, tiles);
}

const char* stencil_name(const char* kind, int prec, int mode, bool fine) {
    // interned names: a node-based set keeps every c_str() pointer stable;
    // batched solves call this from several host threads
    static std::set<std::string>* names = new std::set<std::string>();
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    static const char* precs[3] = {"f64", "f32", "bf16"};
    static const char* modes[kStencilModes] = {"apply", "resid", "jacobi", "jacobi2z"};
    const std::string n = std::string(kind) + "_" + precs[prec] + "_" + modes[mode] + (fine ? "_L0" : "_Lc");
    return names->insert(n).first->c_str();
}

// Algorithmic bytes of one vector-stencil launch: per open face its x and y
// (and f for resid / jacobi; f instead of x for jacobi2z), its A (and 1/D for
// jacobi, jacobi2z), about one edge fraction L and a third of a cell's 1/V.
template <typename T, typename TC>
double vec_stencil_bytes(const Grid3& g, int mode) {
    const double tv = sizeof(T), tc = sizeof(TC);
    const bool jac = mode == ST_JACOBI || mode == ST_JACOBI2Z;
    return (double)g.nopen * (tv * (2 + (mode == ST_RESID || mode == ST_JACOBI)) + tc * (2.0 + 1.0 / 3.0 + jac));
}
// per active cell: x, y (and f), three face fractions (six faces, each shared
// by two cells), 1/D for jacobi, and the activity flag
template <typename T, typename TC>
double scal_stencil_bytes(const Grid3& g, int mode) {
    const double tv = sizeof(T), tc = sizeof(TC);
    return (double)g.nact * (tv * (2 + (mode != ST_APPLY)) + tc * (3 + (mode == ST_JACOBI)) + 1.0);
}

template <typename T, typename TC>
void vec_stencil(const VecOp<T, TC>& op, int mode, const T* x, const T* f, T* y, double omega, cudaStream_t s) {
    const Grid3& g = op.g;
    const double bytes = vec_stencil_bytes<T, TC>(g, mode);
    if (op.tiles) {
        const int* tl = op.stiles ? op.stiles : op.tiles;
        const int nt = op.stiles ? op.nstiles : op.ntiles;
        if (nt <= 0) return;
        const char* nm = stencil_name("vec_stencil", prec_index<T>(), mode, op.level == 0);
        // tile shape: 0 = 32x4x2 (the level's active tiles), 1 = 32x2x4, 2 = 32x8x1; 3 = 32x8x8,
        // 4 = 32x4x8, 5 = 32x8x4 by the z-marching kernel (op.stiles is the active-tile list of that shape)
        switch (op.shape * kStencilModes + mode) {
#define DM_TILED(SH, MD, SY, SZ)                                                                              \
    case SH * kStencilModes + MD:                                                                                         \
        launch_b(nm, bytes, k_vec_stencil_tiled<T, TC, MD, SY, SZ>, nt, dim3(TX, SY, SZ), 0, s, g, op.A, op.L,  \
                 op.invV, op.invD, op.sigma, x, f, y, omega, tl);                                             \
        break;
            DM_TILED(0, ST_APPLY, 4, 2) DM_TILED(0, ST_RESID, 4, 2) DM_TILED(0, ST_JACOBI, 4, 2) DM_TILED(0, ST_JACOBI2Z, 4, 2)
            DM_TILED(1, ST_APPLY, 2, 4) DM_TILED(1, ST_RESID, 2, 4) DM_TILED(1, ST_JACOBI, 2, 4) DM_TILED(1, ST_JACOBI2Z, 2, 4)
            DM_TILED(2, ST_APPLY, 8, 1) DM_TILED(2, ST_RESID, 8, 1) DM_TILED(2, ST_JACOBI, 8, 1) DM_TILED(2, ST_JACOBI2Z, 8, 1)
#undef DM_TILED
#define DM_MARCH(SH, MD, SY, KZ)                                                                                \
    case SH * kStencilModes + MD:                                                                                         \
        launch_b(nm, bytes, k_vec_stencil_march<T, TC, MD, SY, KZ>, nt, dim3(TX, SY, 1), 0, s, g, op.A, op.L,  \
                 op.invV, op.invD, op.sigma, x, f, y, omega, tl);                                             \
        break;
            DM_MARCH(3, ST_APPLY, 8, 8) DM_MARCH(3, ST_RESID, 8, 8) DM_MARCH(3, ST_JACOBI, 8, 8) DM_MARCH(3, ST_JACOBI2Z, 8, 8)
            DM_MARCH(4, ST_APPLY, 4, 8) DM_MARCH(4, ST_RESID, 4, 8) DM_MARCH(4, ST_JACOBI, 4, 8) DM_MARCH(4, ST_JACOBI2Z, 4, 8)
            DM_MARCH(5, ST_APPLY, 8, 4) DM_MARCH(5, ST_RESID, 8, 4) DM_MARCH(5, ST_JACOBI, 8, 4) DM_MARCH(5, ST_JACOBI2Z, 8, 4)
#undef DM_MARCH
            default: throw Error(DM_ERR_INVALID_ARG, "unknown stencil tile shape");
        }
        return;
    }
    if (mode == ST_APPLY)
        launch_b(stencil_name("vec_stencil", prec_index<T>(), ST_APPLY, op.level == 0), bytes, k_vec_stencil<T, TC, ST_APPLY>, tile_grid(g, op.tiles, op.ntiles, 1), kBlock, 0, s, g, op.A, op.L, op.invV, op.invD, op.sigma, x, f, y, omega, op.tiles);
    else if (mode == ST_RESID)
        launch_b(stencil_name("vec_stencil", prec_index<T>(), ST_RESID, op.level == 0), bytes, k_vec_stencil<T, TC, ST_RESID>, tile_grid(g, op.tiles, op.ntiles, 1), kBlock, 0, s, g, op.A, op.L, op.invV, op.invD, op.sigma, x, f, y, omega, op.tiles);
    else if (mode == ST_JACOBI2Z)
        launch_b(stencil_name("vec_stencil", prec_index<T>(), ST_JACOBI2Z, op.level == 0), bytes, k_vec_stencil<T, TC, ST_JACOBI2Z>, tile_grid(g, op.tiles, op.ntiles, 1), kBlock, 0, s, g, op.A, op.L, op.invV, op.invD, op.sigma, x, f, y, omega, op.tiles);
    else
        launch_b(stencil_name("vec_stencil", prec_index<T>(), ST_JACOBI, op.level == 0), bytes, k_vec_stencil<T, TC, ST_JACOBI>, tile_grid(g, op.tiles, op.ntiles, 1), kBlock, 0, s, g, op.A, op.L, op.invV, op.invD, op.sigma, x, f, y, omega, op.tiles);
}

// y = (K - sigma A) x in FP64 over every node of the level (dense grid of
// blocks), launched under a fixed name: makes no host or device allocation.
void vec_apply_dense_f64(const Grid3& g, const double* A, const double* L, const double* invV, double sigma,
                         const double* x, double* y, cudaStream_t s) {
    launch("vec_stencil_f64_apply_noalloc", k_vec_stencil<double, double, ST_APPLY>, node_grid(g), kBlock, 0, s, g, A, L,
           invV, (const double*)nullptr, sigma, x, (const double*)nullptr, y, 0.0, (const int*)nullptr);
}

void band_slots(const Grid3& g, const double* A, const double* L, const double* invV, double sigma, const int* band,
                int nband, double* vals, cudaStream_t s) {
    if (nband <= 0) return;
    launch("k_band_slots", k_band_slots, (nband + 127) / 128, 128, 0, s, g, A, L, invV, sigma, band, nband, vals);
}

template <typename T, typename TC>
void vec_jacobi_zero(const VecOp<T, TC>& op, const T* f, T* y, double omega, cudaStream_t s) {
    const Domain d{op.g, op.tiles, op.ntiles, 3};
    const int blocks = op.tiles ? std::max(op.ntiles, 1) : (int)std::min<long long>((d.len() + 255) / 256, 152 * 16);
    launch_b(stencil_name("jacobi_zero", prec_index<T>(), ST_JACOBI, op.level == 0),
             (double)op.g.nopen * (2.0 * sizeof(T) + sizeof(TC)), k_jacobi_zero<T, TC>, blocks, 256, 0, s, d, op.invD,
             f, y, omega);
}

void vec_diagonal(const Grid3& g, const double* A, const double* L, const double* invV, double sigma, double* d,
                  cudaStream_t s) {
    launch("k_vec_diag", k_vec_diag, node_grid(g), kBlock, 0, s, g, A, L, invV, sigma, d);
}

void vec_dense_assemble(const Grid3& g, const double* A, const double* L, const double* invV, double sigma,
                        const int* list, int n, double* M, cudaStream_t s) {
    if (n <= 0) return;
    launch("k_vec_dense", k_vec_dense, n, 128, 0, s, g, A, L, invV, sigma, list, n, M);
}

template <typename T, typename TC>
void scal_stencil(const ScalOp<T, TC>& op, int mode, const T* x, const T* f, T* y, double omega, cudaStream_t s) {
    const Grid3& g = op.g;
    if (mode == ST_APPLY)
        launch_b(stencil_name("scal_stencil", prec_index<T>(), ST_APPLY, op.level == 0), scal_stencil_bytes<T, TC>(g, ST_APPLY), k_scal_stencil<T, TC, ST_APPLY>, tile_grid(g, op.tiles, op.ntiles, 0), kBlock, 0, s, g, op.A, op.active, op.invD, x, f, y, omega, op.tiles);
    else if (mode == ST_RESID)
        launch_b(stencil_name("scal_stencil", prec_index<T>(), ST_RESID, op.level == 0), scal_stencil_bytes<T, TC>(g, ST_RESID), k_scal_stencil<T, TC, ST_RESID>, tile_grid(g, op.tiles, op.ntiles, 0), kBlock, 0, s, g, op.A, op.active, op.invD, x, f, y, omega, op.tiles);
    else
        launch_b(stencil_name("scal_stencil", prec_index<T>(), ST_JACOBI, op.level == 0), scal_stencil_bytes<T, TC>(g, ST_JACOBI), k_scal_stencil<T, TC, ST_JACOBI>, tile_grid(g, op.tiles, op.ntiles, 0), kBlock, 0, s, g, op.A, op.active, op.invD, x, f, y, omega, op.tiles);
}

template <typename T, typename TC>
void scal_jacobi_zero(const ScalOp<T, TC>& op, const T* f, T* y, double omega, cudaStream_t s) {
    const Domain d{op.g, op.tiles, op.ntiles, 1};
    const int blocks = op.tiles ? std::max(op.ntiles, 1) : (int)std::min<long long>((d.len() + 255) / 256, 152 * 16);
    launch_b(stencil_name("scal_jacobi_zero", prec_index<T>(), ST_JACOBI, op.level == 0),
             (double)op.g.nact * (2.0 * sizeof(T) + sizeof(TC)), k_jacobi_zero<T, TC>, blocks, 256, 0, s, d, op.invD,
             f, y, omega);
}

void scal_diagonal(const Grid3& g, const double* A, const unsigned char* active, double* d, cudaStream_t s) {
    launch("k_scal_diag", k_scal_diag, node_grid(g, 0), kBlock, 0, s, g, A, active, d);
}

void scal_dense_assemble(const Grid3& g, const double* A, const int* list, const unsigned char* pinned, int n,
                         double* M, cudaStream_t s) {
    if (n <= 0) return;
    launch("k_scal_dense", k_scal_dense, n, 128, 0, s, g, A, list, pinned, n, M);
}

void dm_div_a(const Grid3& g, const double* A, const double* x, double* s_out, const int* tiles, int ntiles,
              cudaStream_t s) {
    launch_b("k_div_a", 16.0 * g.nopen + 8.0 * g.nact, k_div_a, tile_grid(g, tiles, ntiles, 0), kBlock, 0, s, g, A, x,
             s_out, tiles);
}

void dm_sub_grad(const Grid3& g, const double* A, const double* x, const double* phi, double* y, const int* tiles,
                 int ntiles, cudaStream_t s) {
    launch_b("k_sub_grad", 24.0 * g.nopen + 8.0 * g.nact, k_sub_grad, tile_grid(g, tiles, ntiles, 1), kBlock, 0, s, g,
             A, x, phi, y, tiles);
}

// explicit instantiations: FP64 storage / FP64 coefficients, FP32 / FP32, BF16 / FP32
#define DM_INST(T, TC)                                                                                          \
    template void vec_stencil<T, TC>(const VecOp<T, TC>&, int, const T*, const T*, T*, double, cudaStream_t);  \
    template void vec_jacobi_zero<T, TC>(const VecOp<T, TC>&, const T*, T*, double, cudaStream_t);            \
    template void scal_stencil<T, TC>(const ScalOp<T, TC>&, int, const T*, const T*, T*, double, cudaStream_t); \
    template void scal_jacobi_zero<T, TC>(const ScalOp<T, TC>&, const T*, T*, double, cudaStream_t);
DM_INST(double, double)
DM_INST(float, float)
DM_INST(__nv_bfloat16, float)
#undef DM_INST

}  // namespace dm
