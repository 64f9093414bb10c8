// Dey--Mittra cut fractions and level bookkeeping on the device.
//
// Sec. 2 (Eq. farInt, Fig. dmFace): l, a = the parts of an edge / face outside
// the conductor; Sec. 5.1 (Eq. divBInt, Fig. dmVol): v = the part of a cell
// outside the conductor; Sec. 6.1: cut volumes from tetrahedral subvolumes that
// conform to the surface.  The surface is the zero set of the piecewise-linear
// interpolant of the nodal level set on the Kuhn split of every cell (6
// tetrahedra sharing the (0,0,0)-(1,1,1) diagonal); its faces are split by
// the diagonal from their lowest to their highest corner.  phi < 0 is vacuum.
//
// This file is compiled without FMA contraction so that sums of fractions
// (and hence the tests 0 < V < 1 that define the smoother band) round the
// same way on every build.
#include "dm_common.cuh"

namespace dm {

namespace {

constexpr int BX = 32, BY = 4, BZ = 2;

__device__ __forceinline__ void cswap(double& a, double& b) {
    double lo = fmin(a, b), hi = fmax(a, b);
    a = lo;
    b = hi;
}

// length fraction of {phi < 0} on a segment
__device__ double seg_frac(double a, double b) {
    const bool na = a < 0.0, nb = b < 0.0;
    if (na == nb) return na ? 1.0 : 0.0;
    return na ? a / (a - b) : b / (b - a);
}

// area fraction of {phi < 0} on a triangle with linear phi
__device__ double tri_frac(double a, double b, double c) {
    cswap(a, b);
    cswap(b, c);
    cswap(a, b);                       // a <= b <= c
    if (a >= 0.0) return 0.0;          // no negative vertex
    if (c < 0.0) return 1.0;           // all negative
    if (b >= 0.0) {                    // one negative vertex: corner triangle
        return (a / (a - b)) * (a / (a - c));
    }
    return 1.0 - (c / (c - a)) * (c / (c - b));   // two negative: whole minus positive corner
}

// volume fraction of {phi < 0} in a tetrahedron with linear phi
__device__ double tet_frac(double a, double b, double c, double d) {
    // sorting network for 4 values
    cswap(a, b);
    cswap(c, d);
    cswap(a, c);
    cswap(b, d);
    cswap(b, c);                       // a <= b <= c <= d
    if (a >= 0.0) return 0.0;
    if (d < 0.0) return 1.0;
    if (b >= 0.0) {                    // one negative vertex (a)
        return (a / (a - b)) * (a / (a - c)) * (a / (a - d));
    }
    if (c >= 0.0) {                    // two negative (a, b): prism split into three tetrahedra
        const double al = a / (a - c), be = a / (a - d), ga = b / (b - c), de = b / (b - d);
        return al * be * (1.0 - de) + al * de * (1.0 - ga) + ga * de;
    }
    // three negative (a, b, c): whole minus the positive corner at d
    return 1.0 - (d / (d - a)) * (d / (d - b)) * (d / (d - c));
}

__device__ __forceinline__ double quad_frac(double c00, double c10, double c01, double c11) {
    return 0.5 * (tri_frac(c00, c10, c11) + tri_frac(c00, c01, c11));
}

// Walls: bit 2a + s of `pmc` set when the wall of axis a (0 x, 1 y, 2 z) on
// side s (0 low, 1 high) is a magnetic symmetry plane, which lies half a cell
// outside the wall's node plane; its normal faces and tangential edges then
// keep their fractions.  Every other wall is a perfect conductor on the node
// plane and closes them.
__device__ __forceinline__ bool closed_on(int pmc, int axis, int idx, int n) {
    return (idx == 0 && !((pmc >> (2 * axis)) & 1)) || (idx == n && !((pmc >> (2 * axis + 1)) & 1));
}

__global__ void k_fractions(Grid3 g, const double* __restrict__ phi, int pmc, double* __restrict__ L,
                            double* __restrict__ A, double* __restrict__ V) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z * BZ + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int p = g.idx(i, j, k);
    const int X = 1, Y = g.sx, Z = g.sxy, N = g.np;
    const double c000 = phi[p];
    const bool wx = closed_on(pmc, 0, i, g.nx), wy = closed_on(pmc, 1, j, g.ny), wz = closed_on(pmc, 2, k, g.nz);
    // edges (closed on conductor walls they are tangential to)
    if (i < g.nx) L[p] = (wy || wz) ? 0.0 : seg_frac(c000, phi[p + X]);
    if (j < g.ny) L[N + p] = (wx || wz) ? 0.0 : seg_frac(c000, phi[p + Y]);
    if (k < g.nz) L[2 * N + p] = (wx || wy) ? 0.0 : seg_frac(c000, phi[p + Z]);
    // faces (corner order: first in-plane axis, then second; closed on conductor walls they are normal to)
    if (j < g.ny && k < g.nz) A[p] = wx ? 0.0 : quad_frac(c000, phi[p + Y], phi[p + Z], phi[p + Y + Z]);
    if (i < g.nx && k < g.nz) A[N + p] = wy ? 0.0 : quad_frac(c000, phi[p + X], phi[p + Z], phi[p + X + Z]);
    if (i < g.nx && j < g.ny) A[2 * N + p] = wz ? 0.0 : quad_frac(c000, phi[p + X], phi[p + Y], phi[p + X + Y]);
    // cell: the 6 Kuhn tetrahedra (0,0,0) -> e_a -> e_a + e_b -> (1,1,1), summed in
    // the order of the permutations (x,y,z), (x,z,y), (y,x,z), (y,z,x), (z,x,y), (z,y,x)
    if (i < g.nx && j < g.ny && k < g.nz) {
        const double c100 = phi[p + X], c010 = phi[p + Y], c001 = phi[p + Z];
        const double c110 = phi[p + X + Y], c101 = phi[p + X + Z], c011 = phi[p + Y + Z];
        const double c111 = phi[p + X + Y + Z];
        double v = 0.0;
        v += tet_frac(c000, c100, c110, c111);
        v += tet_frac(c000, c100, c101, c111);
        v += tet_frac(c000, c010, c110, c111);
        v += tet_frac(c000, c010, c011, c111);
        v += tet_frac(c000, c001, c101, c111);
        v += tet_frac(c000, c001, c011, c111);
        V[p] = v / 6.0;
    }
}

// The outer walls are perfect conductors: normal faces and tangential edges on
// them are closed whatever fractions a caller supplied.
__global__ void k_close_walls(Grid3 g, double* __restrict__ L, double* __restrict__ A) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z * BZ + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int p = g.idx(i, j, k), N = g.np;
    if (i < g.nx && (j == 0 || j == g.ny || k == 0 || k == g.nz)) L[p] = 0.0;
    if (j < g.ny && (i == 0 || i == g.nx || k == 0 || k == g.nz)) L[N + p] = 0.0;
    if (k < g.nz && (i == 0 || i == g.nx || j == 0 || j == g.ny)) L[2 * N + p] = 0.0;
    if (j < g.ny && k < g.nz && (i == 0 || i == g.nx)) A[p] = 0.0;
    if (i < g.nx && k < g.nz && (j == 0 || j == g.ny)) A[N + p] = 0.0;
    if (i < g.nx && j < g.ny && (k == 0 || k == g.nz)) A[2 * N + p] = 0.0;
}

// Sec. 3: faces with 0 < A < a_min are neglected together with their edges.
__global__ void k_neglect(Grid3 g, double a_min, double* __restrict__ L, double* __restrict__ A) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z * BZ + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int p = g.idx(i, j, k);
    const int X = 1, Y = g.sx, Z = g.sxy, N = g.np;
    double a = A[p];
    if (a > 0.0 && a < a_min) {       // x-face: y-edges k, k+1; z-edges j, j+1
        A[p] = 0.0;
        L[N + p] = 0.0; L[N + p + Z] = 0.0; L[2 * N + p] = 0.0; L[2 * N + p + Y] = 0.0;
    }
    a = A[N + p];
    if (a > 0.0 && a < a_min) {       // y-face: x-edges k, k+1; z-edges i, i+1
        A[N + p] = 0.0;
        L[p] = 0.0; L[p + Z] = 0.0; L[2 * N + p] = 0.0; L[2 * N + p + X] = 0.0;
    }
    a = A[2 * N + p];
    if (a > 0.0 && a < a_min) {       // z-face: x-edges j, j+1; y-edges i, i+1
        A[2 * N + p] = 0.0;
        L[p] = 0.0; L[p + Y] = 0.0; L[N + p] = 0.0; L[N + p + X] = 0.0;
    }
}

// Coarse fractions as averages of the fine fractions they cover.
__global__ void k_coarsen(Grid3 gf, Grid3 gc, const double* __restrict__ Lf, const double* __restrict__ Af,
                          const double* __restrict__ Vf, double* __restrict__ Lc, double* __restrict__ Ac,
                          double* __restrict__ Vc) {
    const int I = blockIdx.x * BX + threadIdx.x;
    const int J = blockIdx.y * BY + threadIdx.y;
    const int K = blockIdx.z * BZ + threadIdx.z;
    if (I > gc.nx || J > gc.ny || K > gc.nz) return;
    const int q = gc.idx(I, J, K);
    const int p = gf.idx(2 * I, 2 * J, 2 * K);
    const int X = 1, Y = gf.sx, Z = gf.sxy, N = gf.np, Nc = gc.np;
    if (J < gc.ny && K < gc.nz)
        Ac[q] = 0.25 * (Af[p] + Af[p + Y] + Af[p + Z] + Af[p + Y + Z]);
    if (I < gc.nx && K < gc.nz)
        Ac[Nc + q] = 0.25 * (Af[N + p] + Af[N + p + X] + Af[N + p + Z] + Af[N + p + X + Z]);
    if (I < gc.nx && J < gc.ny)
        Ac[2 * Nc + q] = 0.25 * (Af[2 * N + p] + Af[2 * N + p + X] + Af[2 * N + p + Y] + Af[2 * N + p + X + Y]);
    if (I < gc.nx) Lc[q] = 0.5 * (Lf[p] + Lf[p + X]);
    if (J < gc.ny) Lc[Nc + q] = 0.5 * (Lf[N + p] + Lf[N + p + Y]);
    if (K < gc.nz) Lc[2 * Nc + q] = 0.5 * (Lf[2 * N + p] + Lf[2 * N + p + Z]);
    if (I < gc.nx && J < gc.ny && K < gc.nz) {
        double s = 0.0;
        for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) s += Vf[p + di * X + dj * Y + dk * Z];
        Vc[q] = 0.125 * s;
    }
}

__global__ void k_inv_volume(Grid3 g, const double* __restrict__ V, double* __restrict__ invV) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z * BZ + threadIdx.z;
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;
    const int p = g.idx(i, j, k);
    const double v = V[p];
    invV[p] = v > 0.0 ? 1.0 / v : 0.0;
}

__global__ void k_cut_cells(Grid3 g, const double* __restrict__ V, int* __restrict__ flag) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z * BZ + threadIdx.z;
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;
    const int p = g.idx(i, j, k);
    const double v = V[p];
    flag[p] = (v > 0.0 && v < 1.0) ? 1 : 0;
}

// is any cell in the 26-neighbourhood of cell (i,j,k) cut?
__device__ __forceinline__ bool near_cut(const Grid3& g, const int* __restrict__ flag, int i, int j, int k) {
    for (int dk = -1; dk <= 1; ++dk) {
        const int kk = k + dk;
        if (kk < 0 || kk >= g.nz) continue;
        for (int dj = -1; dj <= 1; ++dj) {
            const int jj = j + dj;
            if (jj < 0 || jj >= g.ny) continue;
            for (int di = -1; di <= 1; ++di) {
                const int ii = i + di;
                if (ii < 0 || ii >= g.nx) continue;
                if (flag[g.idx(ii, jj, kk)]) return true;
            }
        }
    }
    return false;
}

__device__ __forceinline__ bool valid_cell(const Grid3& g, int i, int j, int k) {
    return i >= 0 && j >= 0 && k >= 0 && i < g.nx && j < g.ny && k < g.nz;
}

__global__ void k_band(Grid3 g, const double* __restrict__ A, const int* __restrict__ flag, int* __restrict__ band,
                       int* __restrict__ count) {
    // one block = one 32 x 4 x 2 node block; its band faces are written as one
    // contiguous chunk (node order, x/y/z within a node) so that the sweeps
    // read spatially close faces together
    __shared__ int warp_tot[8];
    __shared__ int base;
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z * BZ + threadIdx.z;
    const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
    const bool node = i <= g.nx && j <= g.ny && k <= g.nz;
    const int p = node ? g.idx(i, j, k) : 0;
    // face of component c at (i,j,k) touches cells (i,j,k) and (i,j,k) - e_c
    const int di[3] = {1, 0, 0}, dj[3] = {0, 1, 0}, dk[3] = {0, 0, 1};
    bool in[3] = {false, false, false};
    int mine = 0;
    if (node) {
        for (int c = 0; c < 3; ++c) {
            if (!(A[c * g.np + p] > 0.0)) continue;
            bool b = false;
            if (valid_cell(g, i, j, k)) b = near_cut(g, flag, i, j, k);
            if (!b && valid_cell(g, i - di[c], j - dj[c], k - dk[c])) b = near_cut(g, flag, i - di[c], j - dj[c], k - dk[c]);
            in[c] = b;
            mine += b ? 1 : 0;
        }
    }
    // block-exclusive prefix of `mine`
    const int lane = tid & 31, wid = tid >> 5;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (tid == 0) {
        int tot = 0;
        for (int w = 0; w < 8; ++w) {
            const int t = warp_tot[w];
            warp_tot[w] = tot;
            tot += t;
        }
        base = tot > 0 ? atomicAdd(count, tot) : 0;
    }
    __syncthreads();
    int slot = base + warp_tot[wid] + incl - mine;
    for (int c = 0; c < 3; ++c)
        if (in[c]) band[slot++] = c * g.np + p;
}

__global__ void k_open_faces(Grid3 g, const double* __restrict__ A, int* __restrict__ list, int* __restrict__ count) {
    // deterministic order (natural): single block walks the grid
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int n = 0;
    for (int c = 0; c < 3; ++c)
        for (int k = 0; k <= g.nz; ++k)
            for (int j = 0; j <= g.ny; ++j)
                for (int i = 0; i <= g.nx; ++i) {
                    const int q = c * g.np + g.idx(i, j, k);
                    if (A[q] > 0.0) list[n++] = q;
                }
    *count = n;
}

__global__ void k_active_cells(Grid3 g, const double* __restrict__ A, int* __restrict__ list,
                               unsigned char* __restrict__ active, int* __restrict__ count, int write_list) {
    // active cell = cell with at least one open face; list in natural order (single thread)
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z * BZ + threadIdx.z;
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;
    const int p = g.idx(i, j, k);
    const int X = 1, Y = g.sx, Z = g.sxy, N = g.np;
    const bool a = A[p] > 0.0 || A[p + X] > 0.0 || A[N + p] > 0.0 || A[N + p + Y] > 0.0 ||
                   A[2 * N + p] > 0.0 || A[2 * N + p + Z] > 0.0;
    active[p] = a ? 1 : 0;
}

__global__ void k_list_active(Grid3 g, const unsigned char* __restrict__ active, int* __restrict__ list,
                              int* __restrict__ count) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int n = 0;
    for (int k = 0; k < g.nz; ++k)
        for (int j = 0; j < g.ny; ++j)
            for (int i = 0; i < g.nx; ++i) {
                const int p = g.idx(i, j, k);
                if (active[p]) list[n++] = p;
            }
    *count = n;
}

// ---- natural <-> padded layouts -------------------------------------------------
// comp: 0..2 faces x,y,z; natural extents per component
struct Ext { int ex, ey, ez; };
__host__ __device__ inline Ext face_ext(const Grid3& g, int c) {
    if (c == 0) return {g.nx + 1, g.ny, g.nz};
    if (c == 1) return {g.nx, g.ny + 1, g.nz};
    return {g.nx, g.ny, g.nz + 1};
}
__host__ __device__ inline Ext edge_ext(const Grid3& g, int c) {
    if (c == 0) return {g.nx, g.ny + 1, g.nz + 1};
    if (c == 1) return {g.nx + 1, g.ny, g.nz + 1};
    return {g.nx + 1, g.ny + 1, g.nz};
}

__global__ void k_pack3(Grid3 g, int edges, double* __restrict__ nat, double* __restrict__ pad, int dir) {
    // dir = 0: natural -> padded; dir = 1: padded -> natural
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z * BZ + threadIdx.z;
    long long base = 0;
    for (int c = 0; c < 3; ++c) {
        const Ext e = edges ? edge_ext(g, c) : face_ext(g, c);
        if (i < e.ex && j < e.ey && k < e.ez) {
            const long long n = base + i + (long long)e.ex * (j + (long long)e.ey * k);
            const int p = c * g.np + g.idx(i, j, k);
            if (dir == 0) pad[p] = nat[n];
            else nat[n] = pad[p];
        }
        base += (long long)e.ex * e.ey * e.ez;
    }
}

__global__ void k_pack1(Grid3 g, int nodes, double* __restrict__ nat, double* __restrict__ pad, int dir) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z * BZ + threadIdx.z;
    const int ex = g.nx + nodes, ey = g.ny + nodes, ez = g.nz + nodes;
    if (i >= ex || j >= ey || k >= ez) return;
    const long long n = i + (long long)ex * (j + (long long)ey * k);
    const int p = g.idx(i, j, k);
    if (dir == 0) pad[p] = nat[n];
    else nat[n] = pad[p];
}

dim3 node_grid(const Grid3& g, int extra = 1) {
    return dim3((g.nx + extra + BX - 1) / BX, (g.ny + extra + BY - 1) / BY, (g.nz + extra + BZ - 1) / BZ);
}
const dim3 kBlock(BX, BY, BZ);

int read_count(const int* d_count, cudaStream_t s) {
    int h = 0;
    DM_CUDA(cudaMemcpyAsync(&h, d_count, sizeof(int), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    return h;
}

}  // namespace

Grid3 make_grid(int nx, int ny, int nz, double hx, double hy, double hz) {
    Grid3 g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.sx = ((nx + 3 + 3) / 4) * 4;
    g.sy = ny + 3;
    g.sz = nz + 3;
    g.sxy = g.sx * g.sy;
    const long long np = (long long)g.sxy * g.sz;
    DM_REQUIRE(np * 3 < (1ll << 31), DM_ERR_INVALID_ARG, "grid too large for 32-bit indexing");
    g.np = (int)np;
    g.off0 = 1 + g.sx * (1 + g.sy);
    g.hx = hx; g.hy = hy; g.hz = hz;
    g.rhx = 1.0 / hx; g.rhy = 1.0 / hy; g.rhz = 1.0 / hz;
    g.rhxf = (float)g.rhx; g.rhyf = (float)g.rhy; g.rhzf = (float)g.rhz;
    return g;
}

long long natural_faces(const Grid3& g) {
    return (long long)(g.nx + 1) * g.ny * g.nz + (long long)g.nx * (g.ny + 1) * g.nz + (long long)g.nx * g.ny * (g.nz + 1);
}
long long natural_edges(const Grid3& g) {
    return (long long)g.nx * (g.ny + 1) * (g.nz + 1) + (long long)(g.nx + 1) * g.ny * (g.nz + 1) +
           (long long)(g.nx + 1) * (g.ny + 1) * g.nz;
}
long long natural_cells(const Grid3& g) { return (long long)g.nx * g.ny * g.nz; }

void geom_fractions(const Grid3& g, const double* phi_pad, int pmc_walls, double* L, double* A, double* V,
                    cudaStream_t s) {
    launch("k_fractions", k_fractions, node_grid(g), kBlock, 0, s, g, phi_pad, pmc_walls, L, A, V);
}

void geom_neglect_faces(const Grid3& g, double a_min, double* L, double* A, cudaStream_t s) {
    launch("k_neglect", k_neglect, node_grid(g), kBlock, 0, s, g, a_min, L, A);
}

void geom_coarsen(const Grid3& gf, const Grid3& gc, const double* Lf, const double* Af, const double* Vf,
                  double* Lc, double* Ac, double* Vc, cudaStream_t s) {
    launch("k_coarsen", k_coarsen, node_grid(gc), kBlock, 0, s, gf, gc, Lf, Af, Vf, Lc, Ac, Vc);
}

void geom_inv_volume(const Grid3& g, const double* V, double* invV, cudaStream_t s) {
    launch("k_inv_volume", k_inv_volume, node_grid(g, 0), kBlock, 0, s, g, V, invV);
}

int geom_band(const Grid3& g, const double* A, const double* V, int* cell_flag, int* band, int* d_count,
              cudaStream_t s) {
    DM_CUDA(cudaMemsetAsync(cell_flag, 0, sizeof(int) * (size_t)g.np, s));
    DM_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int), s));
    launch("k_cut_cells", k_cut_cells, node_grid(g, 0), kBlock, 0, s, g, V, cell_flag);
    launch("k_band", k_band, node_grid(g), kBlock, 0, s, g, A, cell_flag, band, d_count);
    return read_count(d_count, s);
}

__global__ void k_count_positive(long long n, const double* __restrict__ a, int* __restrict__ count) {
    int c = 0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        c += a[r] > 0.0 ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

int count_positive(long long n, const double* a, int* d_count, cudaStream_t s) {
    DM_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int), s));
    const int blocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8));
    launch("k_count_positive", k_count_positive, blocks, 256, 0, s, n, a, d_count);
    return read_count(d_count, s);
}

__global__ void k_count_nonfinite(long long n, const double* __restrict__ a, int* __restrict__ count) {
    int c = 0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        c += isfinite(a[r]) ? 0 : 1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

int count_nonfinite(long long n, const double* a, int* d_count, cudaStream_t s) {
    DM_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int), s));
    const int blocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8));
    launch("k_count_nonfinite", k_count_nonfinite, blocks, 256, 0, s, n, a, d_count);
    return read_count(d_count, s);
}

__global__ void k_count_outside(long long n, const double* __restrict__ a, double lo, double hi,
                                int* __restrict__ count) {
    int c = 0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        c += (a[r] >= lo && a[r] <= hi) ? 0 : 1;   // NaN counts as outside
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

int count_outside(long long n, const double* a, double lo, double hi, int* d_count, cudaStream_t s) {
    DM_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int), s));
    const int blocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8));
    launch("k_count_outside", k_count_outside, blocks, 256, 0, s, n, a, lo, hi, d_count);
    return read_count(d_count, s);
}

__global__ void k_count_flags(long long n, const unsigned char* __restrict__ a, int* __restrict__ count) {
    int c = 0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        c += a[r] ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

int count_flags(long long n, const unsigned char* a, int* d_count, cudaStream_t s) {
    DM_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int), s));
    const int blocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8));
    launch("k_count_flags", k_count_flags, blocks, 256, 0, s, n, a, d_count);
    return read_count(d_count, s);
}

// flags[t] = 1 if tile t holds an open face or an active cell
__global__ void k_tile_flags(Grid3 g, const double* __restrict__ A, const unsigned char* __restrict__ active,
                             int* __restrict__ flags) {
    const int t = blockIdx.x;
    int i0, j0, k0;
    tile_origin(g, t, i0, j0, k0);
    const int i = i0 + (threadIdx.x & (TX - 1)), j = j0 + (threadIdx.x / TX) % TY, k = k0 + threadIdx.x / (TX * TY);
    bool any = false;
    if (i <= g.nx && j <= g.ny && k <= g.nz) {
        const int p = g.idx(i, j, k);
        any = A[p] > 0.0 || A[g.np + p] > 0.0 || A[2 * g.np + p] > 0.0 || active[p] != 0;
    }
    const int v = __syncthreads_or(any);
    if (threadIdx.x == 0) flags[t] = v ? 1 : 0;
}

// out = indices t with flags[t] != 0, ascending (one block of 1024 threads)
__global__ void k_compact(const int* __restrict__ flags, int n, int* __restrict__ out, int* __restrict__ count) {
    __shared__ int scan[1024];
    const int tid = threadIdx.x;
    const int chunk = (n + 1023) / 1024;
    const int b = min(n, tid * chunk), e = min(n, b + chunk);
    int c = 0;
    for (int t = b; t < e; ++t) c += flags[t] != 0;
    scan[tid] = c;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = tid >= o ? scan[tid - o] : 0;
        __syncthreads();
        scan[tid] += v;
        __syncthreads();
    }
    int w = scan[tid] - c;
    for (int t = b; t < e; ++t)
        if (flags[t]) out[w++] = t;
    if (tid == 1023) *count = scan[1023];
}

__global__ void k_tile_flags_shape(Grid3 g, int sy, int sz, const double* __restrict__ A,
                                   const unsigned char* __restrict__ active, int* __restrict__ flags) {
    const int t = blockIdx.x;
    const int nti = (g.nx + TX) / TX, ntj = (g.ny + sy) / sy;
    const int i0 = (t % nti) * TX, j0 = ((t / nti) % ntj) * sy, k0 = (t / (nti * ntj)) * sz;
    bool any = false;
    for (int e = threadIdx.x; e < TX * sy * sz; e += blockDim.x) {
        const int i = i0 + (e & (TX - 1)), j = j0 + (e / TX) % sy, k = k0 + e / (TX * sy);
        if (i <= g.nx && j <= g.ny && k <= g.nz) {
            const int p = g.idx(i, j, k);
            any |= A[p] > 0.0 || A[g.np + p] > 0.0 || A[2 * g.np + p] > 0.0 || active[p] != 0;
        }
    }
    const int v = __syncthreads_or(any);
    if (threadIdx.x == 0) flags[t] = v ? 1 : 0;
}

int geom_tiles_shape(const Grid3& g, int sy, int sz, const double* A, const unsigned char* active, int* tiles,
                     int* flags, int* d_count, cudaStream_t s) {
    const int nt = ((g.nx + TX) / TX) * ((g.ny + sy) / sy) * ((g.nz + sz) / sz);
    launch("k_tile_flags", k_tile_flags_shape, nt, 256, 0, s, g, sy, sz, A, active, flags);
    launch("k_compact", k_compact, 1, 1024, 0, s, flags, nt, tiles, d_count);
    return read_count(d_count, s);
}

int geom_tiles(const Grid3& g, const double* A, const unsigned char* active, int* tiles, int* flags, int* d_count,
               cudaStream_t s) {
    const int nt = tiles_x(g) * tiles_y(g) * tiles_z(g);
    launch("k_tile_flags", k_tile_flags, nt, TX * TY * TZ, 0, s, g, A, active, flags);
    launch("k_compact", k_compact, 1, 1024, 0, s, flags, nt, tiles, d_count);
    return read_count(d_count, s);
}

int geom_open_faces(const Grid3& g, const double* A, int* list, int* d_count, cudaStream_t s) {
    launch("k_open_faces", k_open_faces, 1, 1, 0, s, g, A, list, d_count);
    return read_count(d_count, s);
}

int geom_active_cells(const Grid3& g, const double* A, int* list, unsigned char* active, int* d_count,
                      cudaStream_t s) {
    launch("k_active_cells", k_active_cells, node_grid(g, 0), kBlock, 0, s, g, A, list, active, d_count, 0);
    if (!list) return 0;
    launch("k_list_active", k_list_active, 1, 1, 0, s, g, active, list, d_count);
    return read_count(d_count, s);
}

void pack_nodes(const Grid3& g, const double* nat, double* pad, cudaStream_t s) {
    launch("k_pack1", k_pack1, node_grid(g), kBlock, 0, s, g, 1, const_cast<double*>(nat), pad, 0);
}
void pack_faces(const Grid3& g, const double* nat, double* pad, cudaStream_t s) {
    launch("k_pack3", k_pack3, node_grid(g), kBlock, 0, s, g, 0, const_cast<double*>(nat), pad, 0);
}
void unpack_faces(const Grid3& g, const double* pad, double* nat, cudaStream_t s) {
    launch("k_pack3", k_pack3, node_grid(g), kBlock, 0, s, g, 0, nat, const_cast<double*>(pad), 1);
}
void pack_edges(const Grid3& g, const double* nat, double* pad, cudaStream_t s) {
    launch("k_pack3", k_pack3, node_grid(g), kBlock, 0, s, g, 1, const_cast<double*>(nat), pad, 0);
}
void geom_close_walls(const Grid3& g, double* L, double* A, cudaStream_t s) {
    launch("k_close_walls", k_close_walls, node_grid(g), kBlock, 0, s, g, L, A);
}
void unpack_edges(const Grid3& g, const double* pad, double* nat, cudaStream_t s) {
    launch("k_pack3", k_pack3, node_grid(g), kBlock, 0, s, g, 1, nat, const_cast<double*>(pad), 1);
}
void pack_cells(const Grid3& g, const double* nat, double* pad, cudaStream_t s) {
    launch("k_pack1", k_pack1, node_grid(g, 0), kBlock, 0, s, g, 0, const_cast<double*>(nat), pad, 0);
}
void unpack_cells(const Grid3& g, const double* pad, double* nat, cudaStream_t s) {
    launch("k_pack1", k_pack1, node_grid(g, 0), kBlock, 0, s, g, 0, nat, const_cast<double*>(pad), 1);
}

}  // namespace dm
