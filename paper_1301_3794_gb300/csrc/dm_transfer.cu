// Grid transfers of the geometric V-cycles (a design of this library; the
// paper's multigrid was algebraic, Sec. 6).
//
// Face prolongation P (coarse -> fine, fine grid = 2x coarse), per component:
//   across the face plane: a fine face on a coarse plane copies it, a fine face
//   half-way takes the mean of the two coarse faces around it;
//   within the plane: bilinear, weight 3/4 towards the nearer coarse face
//   centre and 1/4 towards the farther one; at a domain wall the missing
//   neighbour's weight goes to the nearer face.
// The fine result is masked by the open fine faces.  Restriction R = P^T / 8
// is evaluated from the same per-axis weights, masked by the open coarse faces.
//
// Cell transfers: a fine cell copies its parent; R = P^T / 8 (the mean of the
// 8 children); both masked by the active cells of the receiving level.
#include "dm_common.cuh"

namespace dm {

namespace {

constexpr int BX = 32, BY = 4, BZ = 2;
const dim3 kBlock(BX, BY, BZ);

// Fine faces that a coarse face (coarse index c along an axis) gathers, with
// the weights of P^T along that axis: along the face normal the fine planes
// 2c-1, 2c, 2c+1 (weights 1/2, 1, 1/2); within the plane the fine cells
// 2c-1 .. 2c+2 (weights 1/4, 3/4, 3/4, 1/4, the wall rule moving a missing
// neighbour's 1/4 onto the nearer face).  Slots outside the grid get weight 0
// and point at ghost positions (zero in every vector).
__device__ __forceinline__ void restrict_axis(bool normal, int c, int nc, int nf, int idx[4], float w[4]) {
    idx[0] = 2 * c - 1;
    idx[1] = 2 * c;
    idx[2] = 2 * c + 1;
    idx[3] = 2 * c + 2;
    if (normal) {
        w[0] = c >= 1 ? 0.5f : 0.f;
        w[1] = 1.f;
        w[2] = 2 * c + 1 <= nf ? 0.5f : 0.f;
        w[3] = 0.f;
        idx[3] = 2 * c;
    } else {
        const bool lo = c >= 1, hi = c + 1 < nc;
        w[0] = lo ? 0.25f : 0.f;
        w[1] = lo ? 0.75f : 1.f;
        w[2] = hi ? 0.75f : 1.f;
        w[3] = hi ? 0.25f : 0.f;
    }
}

template <typename T, typename TC, bool SYM>
__global__ void k_face_restrict(Grid3 gf, Grid3 gc, const TC* __restrict__ Ac, const T* __restrict__ r,
                                T* __restrict__ fc, const int* __restrict__ tiles) {
    using C = typename Compute<T>::type;
    int I, J, K;
    block_node(gc, tiles, I, J, K);
    if (I > gc.nx || J > gc.ny || K > gc.nz) return;
    const int q = gc.idx(I, J, K);
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        const int oq = comp * gc.np + q;
        C acc = C(0);
        if ((C)Ac[oq] > C(0)) {
            int ix[4], iy[4], iz[4];
            float wx[4], wy[4], wz[4];
            restrict_axis(comp == 0, I, gc.nx, gf.nx, ix, wx);
            restrict_axis(comp == 1, J, gc.ny, gf.ny, iy, wy);
            restrict_axis(comp == 2, K, gc.nz, gf.nz, iz, wz);
            const T* rc = r + comp * gf.np;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                if (comp == 2 && a == 3) continue;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    if (comp == 1 && b == 3) continue;
                    const float wab = wz[a] * wy[b];
                    const T* row = rc + gf.idx(0, iy[b], iz[a]);
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        if (comp == 0 && d == 3) continue;
                        acc += C(wab * wx[d]) * (C)to_c(row[ix[d]]);
                    }
                }
            }
            acc *= C(0.125);
            if (SYM) acc *= sqrt((C)Ac[oq]);
        }
        fc[oq] = to_store<T>(acc);
    }
}

template <typename T, typename TC, bool SYM>
__global__ void k_face_prolong(Grid3 gf, Grid3 gc, const TC* __restrict__ Af, const T* __restrict__ ec,
                               T* __restrict__ x, const int* __restrict__ tiles) {
    using C = typename Compute<T>::type;
    int i, j, k;
    block_node(gf, tiles, i, j, k);
    if (i > gf.nx || j > gf.ny || k > gf.nz) return;
    const int p = gf.idx(i, j, k);
    const int nc[3] = {gc.nx, gc.ny, gc.nz};
    const int f[3] = {i, j, k};
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        const int op = comp * gf.np + p;
        if (!((C)Af[op] > C(0))) continue;
        int ci[3][2];
        float wi[3][2];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const int fi = f[ax];
            if (ax == comp) {
                if ((fi & 1) == 0) { ci[ax][0] = fi >> 1; wi[ax][0] = 1.f; ci[ax][1] = fi >> 1; wi[ax][1] = 0.f; }
                else { ci[ax][0] = fi >> 1; wi[ax][0] = 0.5f; ci[ax][1] = (fi >> 1) + 1; wi[ax][1] = 0.5f; }
            } else {
                const int c = fi >> 1;
                const int nb = (fi & 1) ? c + 1 : c - 1;
                const bool inside = nb >= 0 && nb < nc[ax];
                ci[ax][0] = c; wi[ax][0] = inside ? 0.75f : 1.0f;
                ci[ax][1] = inside ? nb : c; wi[ax][1] = inside ? 0.25f : 0.f;
            }
        }
        C acc = C(0);
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int d = 0; d < 2; ++d) {
                    const float w = wi[2][a] * wi[1][b] * wi[0][d];
                    if (w != 0.f) acc += C(w) * (C)to_c(ec[comp * gc.np + gc.idx(ci[0][d], ci[1][b], ci[2][a])]);
                }
        if (SYM) acc /= sqrt((C)Af[op]);
        x[op] = to_store<T>((C)to_c(x[op]) + acc);
    }
}

// x <- A^(-1/2) x (inverse) or A^(1/2) x on the open faces (closed: 0)
template <typename T, typename TC>
__global__ void k_scale_sqrt_a(Domain d, const TC* __restrict__ A, int inverse, T* __restrict__ x) {
    using C = typename Compute<T>::type;
    for_each_entry(d, [&](long long r) {
        const C a = (C)A[r];
        const C f = a > C(0) ? (inverse ? C(1) / sqrt(a) : sqrt(a)) : C(0);
        x[r] = to_store<T>((C)to_c(x[r]) * f);
    });
}

template <typename T>
__global__ void k_cell_restrict(Grid3 gf, Grid3 gc, const unsigned char* __restrict__ active_c,
                                const T* __restrict__ r, T* __restrict__ fc, const int* __restrict__ tiles) {
    using C = typename Compute<T>::type;
    int I, J, K;
    block_node(gc, tiles, I, J, K);
    if (I >= gc.nx || J >= gc.ny || K >= gc.nz) return;
    const int q = gc.idx(I, J, K);
    C acc = C(0);
    if (active_c[q]) {
        const int p = gf.idx(2 * I, 2 * J, 2 * K);
        for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) acc += (C)to_c(r[p + di + dj * gf.sx + dk * gf.sxy]);
        acc *= C(0.125);
    }
    fc[q] = to_store<T>(acc);
}

template <typename T>
__global__ void k_cell_prolong(Grid3 gf, Grid3 gc, const unsigned char* __restrict__ active_f,
                               const T* __restrict__ ec, T* __restrict__ x, const int* __restrict__ tiles) {
    using C = typename Compute<T>::type;
    int i, j, k;
    block_node(gf, tiles, i, j, k);
    if (i >= gf.nx || j >= gf.ny || k >= gf.nz) return;
    const int p = gf.idx(i, j, k);
    if (!active_f[p]) return;
    x[p] = to_store<T>((C)to_c(x[p]) + (C)to_c(ec[gc.idx(i >> 1, j >> 1, k >> 1)]));
}

inline dim3 grid_for(const Grid3& g, int extra) {
    return dim3((g.nx + extra + BX - 1) / BX, (g.ny + extra + BY - 1) / BY, (g.nz + extra + BZ - 1) / BZ);
}

}  // namespace

template <typename T, typename TC>
void face_restrict(const Grid3& gf, const Grid3& gc, const TC* Ac, const T* r, T* fc, const int* tiles_c,
                   int ntiles_c, cudaStream_t s, bool sym) {
    // every open fine face's r once; per open coarse face its A and f_c
    const double bytes = (double)gf.nopen * sizeof(T) + (double)gc.nopen * (sizeof(T) + sizeof(TC));
    if (sym)
        launch_b("k_face_restrict", bytes, k_face_restrict<T, TC, true>, tile_grid(gc, tiles_c, ntiles_c, 1), kBlock, 0,
                 s, gf, gc, Ac, r, fc, tiles_c);
    else
        launch_b("k_face_restrict", bytes, k_face_restrict<T, TC, false>, tile_grid(gc, tiles_c, ntiles_c, 1), kBlock,
                 0, s, gf, gc, Ac, r, fc, tiles_c);
}
template <typename T, typename TC>
void face_prolong_add(const Grid3& gf, const Grid3& gc, const TC* Af, const T* ec, T* x, const int* tiles_f,
                      int ntiles_f, cudaStream_t s, bool sym) {
    // every open coarse face's e_c once; per open fine face its A and x read and written
    const double bytes = (double)gc.nopen * sizeof(T) + (double)gf.nopen * (2.0 * sizeof(T) + sizeof(TC));
    if (sym)
        launch_b("k_face_prolong", bytes, k_face_prolong<T, TC, true>, tile_grid(gf, tiles_f, ntiles_f, 1), kBlock, 0,
                 s, gf, gc, Af, ec, x, tiles_f);
    else
        launch_b("k_face_prolong", bytes, k_face_prolong<T, TC, false>, tile_grid(gf, tiles_f, ntiles_f, 1), kBlock, 0,
                 s, gf, gc, Af, ec, x, tiles_f);
}
template <typename T, typename TC>
void scale_sqrt_a(const Domain& d, const TC* A, bool inverse, T* x, cudaStream_t s) {
    launch_b("k_scale_sqrt_a", d.live() * (2.0 * sizeof(T) + sizeof(TC)), k_scale_sqrt_a<T, TC>,
             d.tiles ? std::max(d.ntiles, 1) : 1216, 256, 0, s, d, A, inverse ? 1 : 0, x);
}
template <typename T>
void cell_restrict(const Grid3& gf, const Grid3& gc, const unsigned char* active_c, const T* r, T* fc,
                   const int* tiles_c, int ntiles_c, cudaStream_t s) {
    launch_b("k_cell_restrict", (double)gf.nact * sizeof(T) + (double)gc.nact * (sizeof(T) + 1.0), k_cell_restrict<T>,
             tile_grid(gc, tiles_c, ntiles_c, 0), kBlock, 0, s, gf, gc, active_c, r, fc, tiles_c);
}
template <typename T>
void cell_prolong_add(const Grid3& gf, const Grid3& gc, const unsigned char* active_f, const T* ec, T* x,
                      const int* tiles_f, int ntiles_f, cudaStream_t s) {
    launch_b("k_cell_prolong", (double)gc.nact * sizeof(T) + (double)gf.nact * (2.0 * sizeof(T) + 1.0),
             k_cell_prolong<T>, tile_grid(gf, tiles_f, ntiles_f, 0), kBlock, 0, s, gf, gc, active_f, ec, x, tiles_f);
}

#define DM_INST(T, TC)                                                                                   \
    template void face_restrict<T, TC>(const Grid3&, const Grid3&, const TC*, const T*, T*, const int*, int,  \
                                       cudaStream_t, bool);                                                \
    template void face_prolong_add<T, TC>(const Grid3&, const Grid3&, const TC*, const T*, T*, const int*, int, \
                                          cudaStream_t, bool);                                               \
    template void scale_sqrt_a<T, TC>(const Domain&, const TC*, bool, T*, cudaStream_t);
DM_INST(double, double)
DM_INST(float, float)
DM_INST(__nv_bfloat16, float)
#undef DM_INST
template void cell_restrict<double>(const Grid3&, const Grid3&, const unsigned char*, const double*, double*, const int*, int, cudaStream_t);
template void cell_restrict<float>(const Grid3&, const Grid3&, const unsigned char*, const float*, float*, const int*, int, cudaStream_t);
template void cell_restrict<__nv_bfloat16>(const Grid3&, const Grid3&, const unsigned char*, const __nv_bfloat16*,
                                           __nv_bfloat16*, const int*, int, cudaStream_t);
template void cell_prolong_add<double>(const Grid3&, const Grid3&, const unsigned char*, const double*, double*, const int*, int, cudaStream_t);
template void cell_prolong_add<float>(const Grid3&, const Grid3&, const unsigned char*, const float*, float*, const int*, int, cudaStream_t);
template void cell_prolong_add<__nv_bfloat16>(const Grid3&, const Grid3&, const unsigned char*, const __nv_bfloat16*,
                                              __nv_bfloat16*, const int*, int, cudaStream_t);

}  // namespace dm
