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

// weight of coarse index J for fine index jf along an in-plane axis with nc coarse cells
__device__ __forceinline__ float w_inplane(int jf, int J, int nc) {
    const int c = jf >> 1;
    const int nb = (jf & 1) ? c + 1 : c - 1;
    const bool inside = nb >= 0 && nb < nc;
    float w = 0.f;
    if (c == J) w += inside ? 0.75f : 1.0f;
    if (inside && nb == J) w += 0.25f;
    return w;
}
// weight of coarse plane I for fine plane if_ along the face normal
__device__ __forceinline__ float w_normal(int fi, int I) {
    if ((fi & 1) == 0) return (fi >> 1) == I ? 1.0f : 0.0f;
    const int lo = fi >> 1;
    return (lo == I || lo + 1 == I) ? 0.5f : 0.0f;
}

template <typename T, typename TC>
__global__ void k_face_restrict(Grid3 gf, Grid3 gc, const TC* __restrict__ Ac, const T* __restrict__ r,
                                T* __restrict__ fc, const int* __restrict__ tiles) {
    using C = typename Compute<T>::type;
    int I, J, K;
    block_node(gc, tiles, I, J, K);
    if (I > gc.nx || J > gc.ny || K > gc.nz) return;
    const int q = gc.idx(I, J, K);
    const int nc[3] = {gc.nx, gc.ny, gc.nz};
    const int nf[3] = {gf.nx, gf.ny, gf.nz};
    const int cc[3] = {I, J, K};
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        const int oq = comp * gc.np + q;
        C acc = C(0);
        if ((C)Ac[oq] > C(0)) {
            // fine candidates per axis: normal axis 2c-1..2c+1, in-plane 2c-1..2c+2
            int lo[3], hi[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                if (ax == comp) { lo[ax] = max(2 * cc[ax] - 1, 0); hi[ax] = min(2 * cc[ax] + 1, nf[ax]); }
                else { lo[ax] = max(2 * cc[ax] - 1, 0); hi[ax] = min(2 * cc[ax] + 2, nf[ax] - 1); }
            }
            for (int fk = lo[2]; fk <= hi[2]; ++fk) {
                const float wk = comp == 2 ? w_normal(fk, K) : w_inplane(fk, K, nc[2]);
                if (wk == 0.f) continue;
                for (int fj = lo[1]; fj <= hi[1]; ++fj) {
                    const float wj = comp == 1 ? w_normal(fj, J) : w_inplane(fj, J, nc[1]);
                    if (wj == 0.f) continue;
                    for (int fi = lo[0]; fi <= hi[0]; ++fi) {
                        const float wi = comp == 0 ? w_normal(fi, I) : w_inplane(fi, I, nc[0]);
                        if (wi == 0.f) continue;
                        acc += C(wk * wj * wi) * (C)to_c(r[comp * gf.np + gf.idx(fi, fj, fk)]);
                    }
                }
            }
            acc *= C(0.125);
        }
        fc[oq] = to_store<T>(acc);
    }
}

template <typename T, typename TC>
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
        x[op] = to_store<T>((C)to_c(x[op]) + acc);
    }
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
                   int ntiles_c, cudaStream_t s) {
    launch("k_face_restrict", k_face_restrict<T, TC>, tile_grid(gc, tiles_c, ntiles_c, 1), kBlock, 0, s, gf, gc, Ac, r,
           fc, tiles_c);
}
template <typename T, typename TC>
void face_prolong_add(const Grid3& gf, const Grid3& gc, const TC* Af, const T* ec, T* x, const int* tiles_f,
                      int ntiles_f, cudaStream_t s) {
    launch("k_face_prolong", k_face_prolong<T, TC>, tile_grid(gf, tiles_f, ntiles_f, 1), kBlock, 0, s, gf, gc, Af, ec,
           x, tiles_f);
}
template <typename T>
void cell_restrict(const Grid3& gf, const Grid3& gc, const unsigned char* active_c, const T* r, T* fc,
                   const int* tiles_c, int ntiles_c, cudaStream_t s) {
    launch("k_cell_restrict", k_cell_restrict<T>, tile_grid(gc, tiles_c, ntiles_c, 0), kBlock, 0, s, gf, gc,
           active_c, r, fc, tiles_c);
}
template <typename T>
void cell_prolong_add(const Grid3& gf, const Grid3& gc, const unsigned char* active_f, const T* ec, T* x,
                      const int* tiles_f, int ntiles_f, cudaStream_t s) {
    launch("k_cell_prolong", k_cell_prolong<T>, tile_grid(gf, tiles_f, ntiles_f, 0), kBlock, 0, s, gf, gc, active_f,
           ec, x, tiles_f);
}

#define DM_INST(T, TC)                                                                                   \
    template void face_restrict<T, TC>(const Grid3&, const Grid3&, const TC*, const T*, T*, const int*, int,  \
                                       cudaStream_t);                                                      \
    template void face_prolong_add<T, TC>(const Grid3&, const Grid3&, const TC*, const T*, T*, const int*, int, \
                                          cudaStream_t);
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
