// Internal declarations shared by the translation units of libdmeig.
//
// Device layout of one multigrid level ("padded node grid"): every face,
// edge and cell array of the level is indexed by the lower node (i, j, k) of
// its element, in a box with one ghost node on every side:
//     p = off0 + i + sx * (j + sy * k),  i in [-1, nx+1], j in [-1, ny+1], ...
// with sx = round_up(nx + 3, 4), sy = ny + 3, sz = nz + 3, np = sx*sy*sz.
// A face vector is three such blocks [x | y | z] (3*np values); so is an edge
// array.  Positions that are not faces of the grid (ghosts, y-faces at i = nx,
// ...) carry zero coefficients and zero values forever, so every stencil reads
// its +-1 neighbours without bounds checks and every vector operation may run
// over the whole 3*np block.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <type_traits>
#include <utility>
#include <stdexcept>
#include <string>
#include <vector>

#include "dmeig.h"

namespace dm {

struct Error : public std::runtime_error {
    dm_status code;
    Error(dm_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define DM_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            throw ::dm::Error(e_ == cudaErrorMemoryAllocation ? DM_ERR_OOM : DM_ERR_CUDA, \
                              std::string(#call) + ": " + cudaGetErrorString(e_));      \
    } while (0)

#define DM_REQUIRE(cond, code, msg)                      \
    do {                                                 \
        if (!(cond)) throw ::dm::Error((code), (msg));   \
    } while (0)

// Geometry of one level's padded node grid.
struct Grid3 {
    int nx, ny, nz;        // cells
    int sx, sy, sz;        // padded extents (with ghosts)
    int sxy;               // sx * sy
    int np;                // sx * sy * sz, multiple of 4
    int off0;              // index of node (0, 0, 0)
    double hx, hy, hz;     // spacing
    double rhx, rhy, rhz;  // 1 / spacing (computed once on the host, so kernels divide nothing)
    float rhxf, rhyf, rhzf;
    int nopen = 0, nact = 0;   // open faces and active cells of the level (set once counted; byte models)

    __host__ __device__ int idx(int i, int j, int k) const { return off0 + i + sx * (j + sy * k); }
};

Grid3 make_grid(int nx, int ny, int nz, double hx, double hy, double hz);

// 1 / h along axis a in the compute type of a kernel
template <typename C>
__host__ __device__ inline C inv_h(const Grid3& g, int a);
template <>
__host__ __device__ inline double inv_h<double>(const Grid3& g, int a) {
    return a == 0 ? g.rhx : (a == 1 ? g.rhy : g.rhz);
}
template <>
__host__ __device__ inline float inv_h<float>(const Grid3& g, int a) {
    return a == 0 ? g.rhxf : (a == 1 ? g.rhyf : g.rhzf);
}

// Active tiles: 32 x 4 x 2 blocks of node positions (i in [0, nx], ...) that
// hold at least one open face or active cell of the level.  Every vector entry
// outside the active tiles is zero for the life of the level, so kernels walk
// only the tile list.  Tile t sits at (i0, j0, k0) = TX (t % nti), TY ((t / nti)
// % ntj), TZ (t / (nti ntj)) with nti = ceil((nx + 1) / TX), ntj = ceil((ny + 1) / TY).
constexpr int TX = 32, TY = 4, TZ = 2;
__host__ __device__ inline int tiles_x(const Grid3& g) { return (g.nx + TX) / TX; }
__host__ __device__ inline int tiles_y(const Grid3& g) { return (g.ny + TY) / TY; }
__host__ __device__ inline int tiles_z(const Grid3& g) { return (g.nz + TZ) / TZ; }
__host__ __device__ inline void tile_origin(const Grid3& g, int t, int& i0, int& j0, int& k0) {
    const int nti = tiles_x(g), ntj = tiles_y(g);
    i0 = (t % nti) * TX;
    t /= nti;
    j0 = (t % ntj) * TY;
    k0 = (t / ntj) * TZ;
}

// The part of a level's padded arrays a vector kernel visits: the active tiles
// (tiles != nullptr) or the whole array of ncomp * np entries.
struct Domain {
    Grid3 g{};
    const int* tiles = nullptr;
    int ntiles = 0;
    int ncomp = 3;    // 3: face vector, 1: cell vector
    __host__ __device__ long long len() const { return (long long)ncomp * g.np; }
    // entries that can be nonzero: open faces or active cells of a tiled
    // domain, every entry of a flat one (the unit of the byte models)
    double live() const { return tiles ? (double)(ncomp == 3 ? g.nopen : g.nact) : (double)len(); }
};

// Iterate the entries of a domain owned by this thread: calls f(r) for every
// array index r (all components).  Tile mode: block b handles tiles b, b+G, ...
template <class F>
__device__ __forceinline__ void for_each_entry(const Domain& d, F&& f) {
    if (d.tiles) {
        const int tx = threadIdx.x & (TX - 1), ty = (threadIdx.x / TX) & (TY - 1), tz = threadIdx.x / (TX * TY);
        for (int tb = blockIdx.x; tb < d.ntiles; tb += gridDim.x) {
            int i0, j0, k0;
            tile_origin(d.g, d.tiles[tb], i0, j0, k0);
            const int i = i0 + tx, j = j0 + ty, k = k0 + tz;
            if (i > d.g.nx || j > d.g.ny || k > d.g.nz) continue;
            const int p = d.g.idx(i, j, k);
            for (int c = 0; c < d.ncomp; ++c) f((long long)c * d.g.np + p);
        }
    } else {
        const long long n = d.len();
        for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
            f(r);
    }
}


// Node (i, j, k) of this thread in a (TX, TY, TZ) block: from the active tile
// list when there is one, else from a dense 3D grid of blocks.
__device__ __forceinline__ void block_node(const Grid3& g, const int* tiles, int& i, int& j, int& k) {
    if (tiles) {
        int i0, j0, k0;
        tile_origin(g, tiles[blockIdx.x], i0, j0, k0);
        i = i0 + threadIdx.x;
        j = j0 + threadIdx.y;
        k = k0 + threadIdx.z;
    } else {
        i = blockIdx.x * TX + threadIdx.x;
        j = blockIdx.y * TY + threadIdx.y;
        k = blockIdx.z * TZ + threadIdx.z;
    }
}
inline dim3 tile_grid(const Grid3& g, const int* tiles, int ntiles, int extra) {
    if (tiles) return dim3(std::max(ntiles, 1));
    return dim3((g.nx + extra + TX - 1) / TX, (g.ny + extra + TY - 1) / TY, (g.nz + extra + TZ - 1) / TZ);
}

// Stream of the active context: buffers are zero-filled on it, so the fill is
// ordered with the context's kernels whatever kind of stream it is.
extern thread_local cudaStream_t g_stream;
// Launch counter of the active context (kernels this library launched).
extern thread_local long long* g_launch_counter;
inline void count_launch(long long n = 1) {
    if (g_launch_counter) *g_launch_counter += n;
}
void check_launch(const char* what);

// Optional per-kernel timing: with tracing on, every launch is bracketed by a
// pair of CUDA events recorded on the launching stream; elapsed times are
// accumulated per kernel name when the events are resolved.
struct Tracer {
    bool on = false;
    struct Stat {
        std::string name;
        long long launches = 0;
        double ms = 0.0;
        double bytes = 0.0;   // algorithmic bytes of the launches (the launch sites' models; 0 = none)
    };
    std::vector<Stat> stats;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    std::vector<cudaEvent_t> free_events;
    std::vector<cudaEvent_t> all_events;
    cudaEvent_t get_event();
    int stat_index(const char* name);
    void begin(cudaStream_t s, cudaEvent_t* e0, cudaEvent_t* e1);
    void end(const char* name, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double bytes);
    void resolve();
    void reset();
    ~Tracer();
};
extern thread_local Tracer* g_tracer;
// Nonzero while the calling thread issues launches that must not be timed
// (timing creates CUDA events): see UntracedScope.
extern thread_local int g_untraced;
struct UntracedScope {
    UntracedScope() { ++g_untraced; }
    ~UntracedScope() { --g_untraced; }
    UntracedScope(const UntracedScope&) = delete;
    UntracedScope& operator=(const UntracedScope&) = delete;
};

// Launch a kernel on stream s, counting it and (with tracing on) timing it;
// `bytes` is the launch's algorithmic DRAM traffic by the launch site's model
// (what the kernel must read and write at least, counted on the elements that
// can be nonzero), accumulated per kernel name for roofline reports.
template <typename... KArgs, typename... Args>
inline void launch_b(const char* name, double bytes, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t s, Args&&... args) {
    Tracer* t = (g_tracer && g_tracer->on && !g_untraced) ? g_tracer : nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (t) t->begin(s, &e0, &e1);
    kern<<<grid, block, smem, s>>>(std::forward<Args>(args)...);
    if (t) t->end(name, s, e0, e1, bytes);
    count_launch();
    check_launch(name);
}
template <typename... KArgs, typename... Args>
inline void launch(const char* name, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                   Args&&... args) {
    launch_b(name, 0.0, kern, grid, block, smem, s, std::forward<Args>(args)...);
}

// Count of the device memory, pinned host memory, CUDA events and streams the
// library has created in this process (a diagnostic for the calls that
// promise to create none).
void note_allocation();

// Owning device buffer.
template <typename T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    explicit DBuf(size_t count, bool zero = true) { alloc(count, zero); }
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count, bool zero = true) {
        release();
        n = count;
        if (count) {
            note_allocation();
            DM_CUDA(cudaMalloc(&p, count * sizeof(T)));
            if (zero) DM_CUDA(cudaMemsetAsync(p, 0, count * sizeof(T), g_stream));
        }
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    T* get() const { return p; }
};

// ---------------------------------------------------------------------------
// precision helpers
// ---------------------------------------------------------------------------
template <typename T> struct Compute { using type = float; };
template <> struct Compute<double> { using type = double; };

__device__ __forceinline__ double to_c(double v) { return v; }
__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ float to_c(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> __device__ __forceinline__ T from_c(double v);
template <> __device__ __forceinline__ double from_c<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_c<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_c<__nv_bfloat16>(double v) { return __float2bfloat16((float)v); }
template <typename T> __device__ __forceinline__ T from_cf(float v);
template <> __device__ __forceinline__ double from_cf<double>(float v) { return v; }
template <> __device__ __forceinline__ float from_cf<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_cf<__nv_bfloat16>(float v) { return __float2bfloat16(v); }
// store a value computed in the compute type into storage type T
template <typename T> __device__ __forceinline__ T to_store(double v) { return from_c<T>(v); }
template <typename T> __device__ __forceinline__ T to_store(float v) { return from_cf<T>(v); }

// ---------------------------------------------------------------------------
// host-callable kernel wrappers (all issue on `s`)
// ---------------------------------------------------------------------------

// geometry (dm_geometry.cu)
// pmc_walls: bit 2a + s set for a magnetic symmetry plane on the wall of axis a, side s
void geom_fractions(const Grid3& g, const double* phi_pad, int pmc_walls, double* L, double* A, double* V,
                    cudaStream_t s);
void geom_neglect_faces(const Grid3& g, double a_min, double* L, double* A, cudaStream_t s);
void geom_coarsen(const Grid3& gf, const Grid3& gc, const double* Lf, const double* Af, const double* Vf,
                  double* Lc, double* Ac, double* Vc, cudaStream_t s);
void geom_inv_volume(const Grid3& g, const double* V, double* invV, cudaStream_t s);
// returns number of band faces written to `band` (capacity 3*np); `cell_flag` scratch np ints
int geom_band(const Grid3& g, const double* A, const double* V, int* cell_flag, int* band, int* d_count,
              cudaStream_t s);
int geom_open_faces(const Grid3& g, const double* A, int* list, int* d_count, cudaStream_t s);
// number of entries > 0
int count_positive(long long n, const double* a, int* d_count, cudaStream_t s);
// number of entries that are NaN or infinite
int count_nonfinite(long long n, const double* a, int* d_count, cudaStream_t s);
// number of nonzero flags
int count_flags(long long n, const unsigned char* a, int* d_count, cudaStream_t s);
// number of entries outside [lo, hi] (NaN included)
int count_outside(long long n, const double* a, double lo, double hi, int* d_count, cudaStream_t s);
// zero the normal faces and tangential edges on the outer walls
void geom_close_walls(const Grid3& g, double* L, double* A, cudaStream_t s);
// active tiles of a level in ascending order (tiles: capacity of all tiles); returns the count
int geom_tiles(const Grid3& g, const double* A, const unsigned char* active, int* tiles, int* flags, int* d_count,
               cudaStream_t s);
// same for tiles of TX x sy x sz nodes (index t = ti + nti (tj + ntj tk), nti = ceil((nx+1)/TX), ntj = ceil((ny+1)/sy))
int geom_tiles_shape(const Grid3& g, int sy, int sz, const double* A, const unsigned char* active, int* tiles,
                     int* flags, int* d_count, cudaStream_t s);
int geom_active_cells(const Grid3& g, const double* A, int* list, unsigned char* active, int* d_count,
                      cudaStream_t s);
// natural <-> padded layouts
void pack_nodes(const Grid3& g, const double* nat, double* pad, cudaStream_t s);
void pack_faces(const Grid3& g, const double* nat, double* pad, cudaStream_t s);
void pack_edges(const Grid3& g, const double* nat, double* pad, cudaStream_t s);
void unpack_faces(const Grid3& g, const double* pad, double* nat, cudaStream_t s);
void unpack_edges(const Grid3& g, const double* pad, double* nat, cudaStream_t s);
void pack_cells(const Grid3& g, const double* nat, double* pad, cudaStream_t s);
void unpack_cells(const Grid3& g, const double* pad, double* nat, cudaStream_t s);
long long natural_faces(const Grid3& g);
long long natural_edges(const Grid3& g);
long long natural_cells(const Grid3& g);

// vector stencils (dm_stencil.cu); T = storage, TC = coefficient type
template <typename T, typename TC>
struct VecOp {
    Grid3 g;
    const TC* A;     // 3*np face fractions
    const TC* L;     // 3*np edge fractions
    const TC* invV;  // np inverse cell fractions (0 where V = 0)
    const TC* invD;  // 3*np inverse diagonal of K - sigma A (0 on closed faces)
    double sigma;
    int level = 0;   // multigrid level (names the kernel in traces: fine vs coarse)
    const int* tiles = nullptr;   // active tiles of the level (nullptr: whole grid)
    int ntiles = 0;
    // tile list and shape used by the tiled vector stencil (chosen by the
    // autotuner; by default the 32x4x2 active tiles above)
    const int* stiles = nullptr;
    int nstiles = 0;
    int shape = 0;
};
// tile shapes of the vector stencil: TX x SY x SZ with (SY, SZ) = (4,2), (2,4), (8,1) (one node per
// thread) and (8,8), (4,8), (8,4) (z-marching: a TX x SY block walks SZ planes)
constexpr int kStencilShapes = 6;
inline void stencil_shape_dims(int shape, int& sy, int& sz) {
    static const int d[kStencilShapes][2] = {{4, 2}, {2, 4}, {8, 1}, {8, 8}, {4, 8}, {8, 4}};
    sy = d[shape][0];
    sz = d[shape][1];
}
enum StencilMode { ST_APPLY = 0, ST_RESID = 1, ST_JACOBI = 2, ST_JACOBI2Z = 3 };
constexpr int kStencilModes = 4;
// trace name of a stencil launch: "<kind>_<precision>_<mode>_<L0|Lc>"
template <typename T> constexpr int prec_index() {
    return std::is_same<T, double>::value ? 0 : (std::is_same<T, float>::value ? 1 : 2);
}
const char* stencil_name(const char* kind, int prec, int mode, bool fine);
// mode APPLY: y = (K - sigma A) x;  RESID: y = f - (K - sigma A) x;
// JACOBI: y = x + omega invD (f - (K - sigma A) x);  JACOBI2Z: two JACOBI
// sweeps from x = 0, the first one's iterate omega invD f (rounded to T as
// vec_jacobi_zero stores it) formed where the second one loads x (x unused)
template <typename T, typename TC>
void vec_stencil(const VecOp<T, TC>& op, int mode, const T* x, const T* f, T* y, double omega, cudaStream_t s);
template <typename T, typename TC>
void vec_jacobi_zero(const VecOp<T, TC>& op, const T* f, T* y, double omega, cudaStream_t s);
// The couplings of one face row of K - sigma A (a face of component c at node
// p) sit in 15 fixed slots: slot 0 the face itself, 1..6 the same component at
// -e_x, +e_x, -e_y, +e_y, -e_z, +e_z; 7..10 component (c+1)%3 and 11..14
// component (c+2)%3, each at offset -1 or 0 along axis c and 0 or +1 along the
// column's own axis.
constexpr int kBandSlots = 15;
// copy code of an empty lane in the band smoother's warp groups
constexpr int kDummyCopy = -2147483647 - 1;
__host__ __device__ inline void band_slot(int c, int e, int& cc, int o[3]) {
    o[0] = o[1] = o[2] = 0;
    if (e < 7) {
        cc = c;
        if (e > 0) o[(e - 1) >> 1] = ((e - 1) & 1) ? 1 : -1;
    } else {
        const int k = (e - 7) & 3;
        cc = (c + 1 + (e - 7) / 4) % 3;
        o[c] = (k >> 1) ? 0 : -1;
        o[cc] = k & 1;
    }
}
// offset of slot e's column from the row's packed index (padded layout)
__host__ __device__ inline int band_slot_offset(int c, int e, int np, int sx, int sxy) {
    int cc, o[3];
    band_slot(c, e, cc, o);
    return (cc - c) * np + o[0] + o[1] * sx + o[2] * sxy;
}
// 15 slot coefficients of every band row (slot-major, FP64)
void band_slots(const Grid3& g, const double* A, const double* L, const double* invV, double sigma, const int* band,
                int nband, double* vals, cudaStream_t s);

// Subdomains of the band smoother (dm_band.cu).  Host form: copies of band
// faces grouped by brick (off), each copy's band position (copy; -1 - t when
// the brick does not own it) and its position in the subdomain's local box of
// nodes (pos = ((c lz + k) ly + j) lx + i, box dims packed in dims).
// Subdomains are stored class by class (schwarz_class of their row count):
// class k holds subdomains cls_first[k] .. cls_first[k] + cls_count[k] - 1.
constexpr int kSchwarzClasses = 5;
int schwarz_class(int rows);
struct SchwarzLayout {
    std::vector<int> off, copy, pos, dims;
    std::vector<int> org;         // 3 per subdomain: node coordinates of its local box's first node
    int maxrows = 0, maxbox = 0;
    bool fixed = false;           // every subdomain uses the fixed box of the default brick
    int cls_first[kSchwarzClasses] = {}, cls_count[kSchwarzClasses] = {};
    long long cls_copies[kSchwarzClasses] = {}, cls_owned[kSchwarzClasses] = {};   // row copies, owned ones
};
template <typename TC>
struct BandSchwarz {
    const int* off = nullptr;
    const int* copy = nullptr;
    const int* pos = nullptr;
    const int* dims = nullptr;
    const int* org = nullptr;
    const TC* vals = nullptr;     // [15][ncopies] slot coefficients of each copy's row
    int nsub = 0, ncopies = 0, maxrows = 0, maxbox = 0;
    int cls_first[kSchwarzClasses] = {}, cls_count[kSchwarzClasses] = {};
    long long cls_copies[kSchwarzClasses] = {}, cls_owned[kSchwarzClasses] = {};
    bool fixed = false;
};
void band_schwarz_setup(const Grid3& g, const int* band_dev, int nband, int brick, SchwarzLayout& out,
                        cudaStream_t s);
// per-copy slot coefficients from the band rows' (both slot-major)
void band_copy_vals(const int* copy, int ncopies, const double* band_vals, int nband, double* out, cudaStream_t s);
// checks the shared-memory need of the largest subdomain box and enables it
template <typename T, typename TC>
void band_schwarz_prepare(const SchwarzLayout& sl);
// x <- x + (restricted additive Schwarz correction on the band); u: nband doubles of scratch
// Streams and events that let the band smoother's class launches run side by
// side (they read the same x and f and write disjoint parts of u): the classes
// after the first go on aux[0 .. naux-1], forked from and joined back into the
// calling stream with the events (in a stream capture these become parallel
// branches of the graph).  naux = 0 launches every class on the calling stream.
constexpr int kForkStreams = kSchwarzClasses - 1;
struct Fork {
    int naux = 0;
    cudaStream_t aux[kForkStreams] = {};
    cudaEvent_t fork = nullptr, join[kForkStreams] = {};
};
template <typename T, typename TC>
void band_schwarz(const BandSchwarz<TC>& bs, const TC* invD, const Grid3& g, const int* band, int nband, const T* f,
                  T* x, double* u, double omega, int sweeps, bool fine, cudaStream_t s, const Fork* fk = nullptr);
void vec_apply_dense_f64(const Grid3& g, const double* A, const double* L, const double* invV, double sigma,
                         const double* x, double* y, cudaStream_t s);
// (K - sigma A) x in float-float into the compact vector out (out[cmap[q]] for
// the open faces q), over the level's 32 x 4 x 2 active tiles; A, L, invV:
// float-float copies of the level's coefficients (to_ff)
void vec_apply_ff(const Grid3& g, const int* tiles, int ntiles, const float2* A, const float2* L, const float2* invV,
                  double sigma, const double* x, const int* cmap, float2* out, cudaStream_t s);
void to_ff(long long n, const double* a, float2* out, cudaStream_t s);
// D A D^T x in float-float into the compact vector out (out[cmap[p]] for the
// active cells p), over the level's active tiles; A: float-float face fractions
void scal_apply_ff(const Grid3& g, const int* tiles, int ntiles, const float2* A, const double* x, const int* cmap,
                   float2* out, cudaStream_t s);
// cmap[q] = position of q in the ascending list (nl entries), -1 elsewhere (n3 entries)
void compact_map(long long n3, const int* list, int nl, int* cmap, cudaStream_t s);
void vec_diagonal(const Grid3& g, const double* A, const double* L, const double* invV, double sigma, double* d,
                  cudaStream_t s);
void vec_dense_assemble(const Grid3& g, const double* A, const double* L, const double* invV, double sigma,
                        const int* list, int n, double* M, cudaStream_t s);

// scalar (cell) stencils: S = D A D^T
template <typename T, typename TC>
struct ScalOp {
    Grid3 g;
    const TC* A;                    // 3*np
    const unsigned char* active;    // np
    const TC* invD;                 // np
    int level = 0;
    const int* tiles = nullptr;
    int ntiles = 0;
};
template <typename T, typename TC>
void scal_stencil(const ScalOp<T, TC>& op, int mode, const T* x, const T* f, T* y, double omega, cudaStream_t s);
template <typename T, typename TC>
void scal_jacobi_zero(const ScalOp<T, TC>& op, const T* f, T* y, double omega, cudaStream_t s);
void scal_diagonal(const Grid3& g, const double* A, const unsigned char* active, double* d, cudaStream_t s);
void scal_dense_assemble(const Grid3& g, const double* A, const int* list, const unsigned char* pinned, int n,
                         double* M, cudaStream_t s);
// divergence s = D (A x) and gradient correction y = x - D^T phi (masked)
void dm_div_a(const Grid3& g, const double* A, const double* x, double* s_out, const int* tiles, int ntiles,
              cudaStream_t s);
void dm_sub_grad(const Grid3& g, const double* A, const double* x, const double* phi, double* y, const int* tiles,
                 int ntiles, cudaStream_t s);

// transfers (dm_transfer.cu)
// tiles_c / tiles_f: active tiles of the level written (nullptr: whole grid)
// sym: the transfers of Eq. fullMat2's congruence form (b~ = A^1/2 b on every
// level): restriction A_c^1/2 R A^-1/2 (the fine input must come pre-scaled by
// A^-1/2, see scale_sqrt_a; the kernel applies A_c^1/2), prolongation
// A^-1/2 P A_c^1/2 (the coarse input must come pre-scaled by A_c^1/2; the
// kernel applies A^-1/2)
template <typename T, typename TC>
void face_restrict(const Grid3& gf, const Grid3& gc, const TC* Ac, const T* r, T* fc, const int* tiles_c,
                   int ntiles_c, cudaStream_t s, bool sym = false);
template <typename T, typename TC>
void face_prolong_add(const Grid3& gf, const Grid3& gc, const TC* Af, const T* ec, T* x, const int* tiles_f,
                      int ntiles_f, cudaStream_t s, bool sym = false);
// x <- A^-1/2 x (inverse) or A^1/2 x on the open faces of the domain
template <typename T, typename TC>
void scale_sqrt_a(const Domain& d, const TC* A, bool inverse, T* x, cudaStream_t s);
template <typename T>
void cell_restrict(const Grid3& gf, const Grid3& gc, const unsigned char* active_c, const T* r, T* fc,
                   const int* tiles_c, int ntiles_c, cudaStream_t s);
template <typename T>
void cell_prolong_add(const Grid3& gf, const Grid3& gc, const unsigned char* active_f, const T* ec, T* x,
                      const int* tiles_f, int ntiles_f, cudaStream_t s);

// dense (dm_dense.cu)
// in-place inverse of the n x n row-major FP64 matrix M (work: 2 n^2 + n doubles).
// Returns false if a pivot fell below tiny * max|M|.
bool dense_inverse(double* M, int n, double* work, int* d_flag, cudaStream_t s);
template <typename T>
void dense_coarse_solve(const double* Minv64, const float* Minv32, int n, const int* list, const unsigned char* zero_rows,
                        const T* f, T* x, double* tmp_in, double* tmp_out, cudaStream_t s);
// connected components of active coarsest cells: pinned[c] = 1 for the lowest
// index of every component (list order = natural order)
void cell_components_pin(const Grid3& g, const double* A, const int* list, int n, int* label,
                         unsigned char* pinned, cudaStream_t s);

// BLAS-1 style (dm_blas.cu); all FP64 unless templated
struct Reducer {
    double* partial = nullptr;   // device, cap_blocks * max_cols
    double* result = nullptr;    // device, max_cols
    double* host = nullptr;      // pinned host, max_cols
    int cap_blocks = 0, max_cols = 0;
};
void reducer_init(Reducer& r, int max_cols);
void reducer_free(Reducer& r);
// sum of x[q] y[q] (times w[q], w nullable = 1) over the n listed indices (host result)
double dot_list(Reducer& red, long long n, const int* list, const double* x, const double* y, const double* w,
                cudaStream_t s);
// out[c] = sum_r w[r] * V[c*ld + r] * x[r] over the domain (w nullable = 1), c < m; result copied to host
void mdot(Reducer& red, const Domain& d, int m, const double* V, long long ld, const double* x, const double* w,
          double* host_out, cudaStream_t s);
// as mdot, and also returns sum_r w[r] x[r]^2 in *self_out (one pass, one sync)
void mdot_self(Reducer& red, const Domain& d, int m, const double* V, long long ld, const double* x, const double* w,
               double* host_out, double* self_out, cudaStream_t s);
// x -= sum_c h[c] V[c*ld + r] using the h the preceding mdot left on the device (red.result),
// and returns sum_r w[r] x[r]^2 of the updated x (one pass, one sync)
// Ascending list of the indices r < n with x[r] > 0 (ordered compaction);
// returns its length.
template <typename T>
int list_flagged(long long n, const T* x, DBuf<int>& out, cudaStream_t s);
// Compact float-float vectors over an index list: y[i] = split(a x[list[i]]);
// y[list[i]] = a x[i] in storage type T (other entries of y untouched).
void ff_gather(long long n, const int* list, double a, const double* x, float2* y, cudaStream_t s);
template <typename T>
void ff_scatter(long long n, const int* list, double a, const float2* x, T* y, cudaStream_t s);
// Delayed classical Gram-Schmidt (DCGS2) on float-float vectors: Q = the j
// finished basis vectors, v = the pending vector, w = the new one.
//   dcgs_dots: out = [Q^T v (j), Q^T w (j), v.v, v.w] (one pass, one sync)
//   dcgs_update: with coef = [s (j), gamma (j), 1/beta, delta]:
//     v <- (v - Q s) / beta,  out <- w - Q gamma - delta v_old;  returns |out|^2
void dcgs_dots(Reducer& red, const Domain& d, int j, const float2* Q, long long ld, const float2* v, const float2* w,
               double* host_out, cudaStream_t s);
double dcgs_update(Reducer& red, const Domain& d, int j, const float2* Q, long long ld, const double* coef_host,
                   float2* v, const float2* w, float2* out, cudaStream_t s);
double maxpy_norm(Reducer& red, const Domain& d, int m, const double* V, long long ld, double* x, const double* w,
                  cudaStream_t s);
// x -= sum_c h[c] V[c*ld + r]    (h host array, m <= max_cols)
void maxpy(Reducer& red, const Domain& d, int m, const double* V, long long ld, const double* h_host, double* x,
           cudaStream_t s);
// out_j = sum_c V_c * Y[c + ldy*j]  for j < p  (Y device, m x p column-major), out may not alias V
void vgemm(const Domain& d, int m, int p, const double* V, long long ld, const double* Y_dev, int ldy, double* out,
           long long ldo, cudaStream_t s);
void axpby(const Domain& d, double a, const double* x, double b, double* y, cudaStream_t s);  // y = a x + b y
void scale_copy(const Domain& d, double a, const double* x, double* y, cudaStream_t s);         // y = a x
void hadamard(const Domain& d, const double* a, const double* x, double* y, cudaStream_t s);    // y = a .* x
template <typename TD, typename TS>
void convert(const Domain& d, const TS* x, TD* y, cudaStream_t s);
template <typename TD>
void convert_coeff(long long n, const double* x, TD* y, cudaStream_t s);
void fill_random(const Domain& d, unsigned long long seed, const double* mask, double* x, cudaStream_t s);
void zero(void* p, size_t bytes, cudaStream_t s);

// FMA issue rates of the current device in FP64 and FP32, flop/s (dm_probe.cu)
void probe_fma_rates(cudaStream_t s, double* fp64_flops, double* fp32_flops);

}  // namespace dm
