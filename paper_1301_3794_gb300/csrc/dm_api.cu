// C ABI and host orchestration of the Dey--Mittra eigensolver (include/dmeig.h).
//
// The host code only sequences kernels and does O(m^2) arithmetic on scalars
// the device returns (Givens rotations of FGMRES, the <= 64 x 64 projected
// eigenproblem of Krylov--Schur); every vector operation runs in the kernels
// of dm_geometry.cu, dm_stencil.cu, dm_transfer.cu, dm_blas.cu, dm_dense.cu.
#include "dm_common.cuh"
#include "dm_learned.cuh"

#include <array>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <atomic>
#include <memory>
#include <mutex>
#include <thread>
#include <numeric>
#include <random>

namespace dm {

thread_local long long* g_launch_counter = nullptr;
thread_local cudaStream_t g_stream = nullptr;
thread_local Tracer* g_tracer = nullptr;
thread_local int g_untraced = 0;

static std::atomic<long long> g_allocations{0};
void note_allocation() { g_allocations.fetch_add(1, std::memory_order_relaxed); }

cudaEvent_t Tracer::get_event() {
    if (free_events.empty()) {
        cudaEvent_t e;
        note_allocation();
        DM_CUDA(cudaEventCreate(&e));
        all_events.push_back(e);
        return e;
    }
    cudaEvent_t e = free_events.back();
    free_events.pop_back();
    return e;
}
int Tracer::stat_index(const char* name) {
    for (size_t i = 0; i < stats.size(); ++i)
        if (stats[i].name == name) return (int)i;
    stats.push_back(Stat{name, 0, 0.0, 0.0});
    return (int)stats.size() - 1;
}
void Tracer::begin(cudaStream_t s, cudaEvent_t* e0, cudaEvent_t* e1) {
    if (pending.size() >= 4096) resolve();
    *e0 = get_event();
    *e1 = get_event();
    DM_CUDA(cudaEventRecord(*e0, s));
}
void Tracer::end(const char* name, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double bytes) {
    DM_CUDA(cudaEventRecord(e1, s));
    const int i = stat_index(name);
    stats[i].bytes += bytes;
    pending.push_back({i, {e0, e1}});
}
void Tracer::resolve() {
    for (auto& p : pending) {
        DM_CUDA(cudaEventSynchronize(p.second.second));
        float ms = 0.f;
        DM_CUDA(cudaEventElapsedTime(&ms, p.second.first, p.second.second));
        stats[p.first].launches += 1;
        stats[p.first].ms += ms;
        free_events.push_back(p.second.first);
        free_events.push_back(p.second.second);
    }
    pending.clear();
}
void Tracer::reset() {
    resolve();
    stats.clear();
}
Tracer::~Tracer() {
    for (auto& p : pending) {
        (void)p;
    }
    for (cudaEvent_t e : all_events) cudaEventDestroy(e);
}

void check_launch(const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(DM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool can_coarsen(int nx, int ny, int nz, int max_coarse) {
    return nx % 2 == 0 && ny % 2 == 0 && nz % 2 == 0 && std::max(nx, std::max(ny, nz)) > max_coarse &&
           std::min(nx, std::min(ny, nz)) >= 4;
}

}  // namespace dm

using namespace dm;

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
struct dm_context {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    long long launches = 0;
    Reducer red;
    Tracer tracer;
    // autotuner cache: (nx, ny, nz, precision) -> stencil tile shape
    std::vector<std::pair<std::array<int, 4>, int>> tuned;
};

namespace {

struct GeoLevel {
    Grid3 g{};
    DBuf<double> A, L, V, invV;
    DBuf<float> A32, L32, invV32;
    DBuf<int> band;
    int nband = 0;
    DBuf<unsigned char> active;
    int nopen = 0;       // open faces (counted once at creation)
    DBuf<int> tiles;     // active tiles (ascending)
    int ntiles = 0;
    Domain vdom() const { return Domain{g, tiles.get(), ntiles, 3}; }   // face vectors
    Domain sdom() const { return Domain{g, tiles.get(), ntiles, 1}; }   // cell vectors
    // ascending lists of the open faces and the active cells (the compact index
    // spaces of the Krylov bases); built with the first operator on the level
    DBuf<int> flist, clist;
    int nflist = -1, nclist = -1;
    // float-float copies of A, L, 1/V and the padded-to-compact face map, for
    // the float-float operator apply of the shifted solves (fine level only,
    // built with the first operator that asks for them)
    DBuf<float2> ffA, ffL, ffV;
    DBuf<int> fmap, fmapc;   // padded-to-compact maps of the open faces and of the active cells
    bool ff = false;
};

struct Sync {
    static void stream(cudaStream_t s) { DM_CUDA(cudaStreamSynchronize(s)); }
};

struct LaunchScope {
    long long* prev;
    Tracer* prev_t;
    cudaStream_t prev_s;
    explicit LaunchScope(dm_context* ctx) : prev(g_launch_counter), prev_t(g_tracer), prev_s(g_stream) {
        g_launch_counter = ctx ? &ctx->launches : nullptr;
        g_tracer = ctx ? &ctx->tracer : nullptr;
        g_stream = ctx ? ctx->stream : nullptr;
    }
    ~LaunchScope() {
        g_launch_counter = prev;
        g_tracer = prev_t;
        g_stream = prev_s;
    }
};

template <class F>
dm_status guarded(const dm_context* cctx, F&& f) {
    dm_context* ctx = const_cast<dm_context*>(cctx);
    LaunchScope scope(ctx);
    try {
        f();
        if (ctx) ctx->err.clear();
        return DM_OK;
    } catch (const Error& e) {
        if (ctx) ctx->err = e.what();
        return e.code;
    } catch (const std::bad_alloc&) {
        if (ctx) ctx->err = "host allocation failed";
        return DM_ERR_OOM;
    } catch (const std::exception& e) {
        if (ctx) ctx->err = e.what();
        return DM_ERR_CUDA;
    } catch (...) {
        if (ctx) ctx->err = "unknown error";
        return DM_ERR_CUDA;
    }
}

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// symmetric eigenproblem of a small dense matrix by cyclic Jacobi rotations
// (a: n x n row-major, destroyed; w: eigenvalues; v: eigenvectors as columns)
void jacobi_eig(int n, std::vector<double>& a, std::vector<double>& w, std::vector<double>& v) {
    v.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
    double scale = 0.0;
    for (double x : a) scale = std::max(scale, std::fabs(x));
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += a[(size_t)p * n + q] * a[(size_t)p * n + q];
        if (std::sqrt(off) <= 1e-17 * std::max(scale, 1e-300)) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
                const double tau = (aqq - app) / (2.0 * apq);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
                    v[(size_t)k * n + p] = c * vkp - s * vkq;
                    v[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = a[(size_t)i * n + i];
}

}  // namespace

struct dm_learned {
    dm_context* ctx = nullptr;
    LearnedNet net;
};

struct dm_geometry {
    dm_context* ctx = nullptr;
    std::vector<std::unique_ptr<GeoLevel>> lv;
    std::mutex mu;   // guards the lazily made FP32 coefficient copies
};

namespace {

// buffers of one level of the V-cycles, in the preconditioner's storage type
struct WorkLevel {
    DBuf<char> f, e, r;       // vector (3 np)
    DBuf<char> sf, se, sr;    // scalar (np)
};

struct OpLevel {
    DBuf<double> invD;        // 3 np
    DBuf<float> invD32;
    DBuf<double> invDs;       // np
    DBuf<float> invDs32;
    double omega = 0.0, omega_s = 0.0;
    int shape = 0;            // stencil tile shape (autotuned)
    DBuf<int> stiles;         // active tiles of that shape (shape != 0)
    int nstiles = 0;
    // subdomains of the band smoother (see dm_band.cu) and their rows' slot coefficients
    DBuf<int> sd_off, sd_copy, sd_pos, sd_dims, sd_org;
    DBuf<double> sd_v64;
    DBuf<float> sd_v32;
    int sd_nsub = 0, sd_ncopies = 0, sd_maxrows = 0, sd_maxbox = 0;
    int sd_cls_first[kSchwarzClasses] = {}, sd_cls_count[kSchwarzClasses] = {};
    long long sd_cls_copies[kSchwarzClasses] = {}, sd_cls_owned[kSchwarzClasses] = {};
    bool sd_fixed = false;
};

// FGMRES workspace: the Arnoldi basis V and the work vector wf in
// float-float (see dcgs_dots), the preconditioned vectors Z and the operator
// output w in FP64
struct Fgmres {
    long long n = 0, nc = 0;   // padded vector length, compact (basis) length
    int m = 0;
    DBuf<float2> V, wf;
    DBuf<double> Z, w;
    void ensure(long long n_, long long nc_, int m_) {
        if (n == n_ && nc == nc_ && m >= m_) return;
        n = n_;
        nc = nc_;
        m = m_;
        V.alloc((size_t)(m + 1) * nc);
        wf.alloc((size_t)nc);
        Z.alloc((size_t)m * n);
        w.alloc((size_t)n);
    }
};

}  // namespace

struct dm_operator {
    dm_context* ctx = nullptr;
    const dm_geometry* geom = nullptr;
    double sigma = 0.0;
    dm_mg_params mg{};
    int nlev = 0;
    std::vector<OpLevel> ol;
    std::vector<WorkLevel> wk;
    DBuf<double> band_u;
    // coarsest vector solve
    DBuf<int> c_list;
    int c_n = 0;
    DBuf<double> c_inv, c_tmp_in, c_tmp_out;
    DBuf<float> c_inv32;
    // coarsest scalar solve
    DBuf<int> s_list;
    int s_n = 0;
    DBuf<unsigned char> s_pinned;
    DBuf<double> s_inv, s_tmp_in, s_tmp_out;
    DBuf<float> s_inv32;
    // FP64 scratch on the fine level
    DBuf<double> t0, t1, t2, t3, c0, c1;
    Fgmres vg, sg;
    double complexity = 1.0;
    // V-cycles captured as CUDA graphs (level-0 work buffers as fixed input/output)
    cudaGraphExec_t vexec = nullptr, sexec = nullptr;
    long long vexec_kernels = 0, sexec_kernels = 0;
    int vcalls = 0, scalls = 0;
    bool graphs = true;
    // learned correction after the V-cycle (own copy of the network's weights and buffers)
    std::unique_ptr<LearnedNet> lnet;
    DBuf<char> lc_c, lc_kc;        // its correction and the operator applied to it
    DBuf<double> lc_part;
    std::vector<double> lc_host;
    bool learned_active = false;
    int learned_applied = 0, learned_fallbacks = 0;
    int learned_streak = 0;    // consecutive shifted solves in which the correction was switched off
    long long nopen0 = 0;
    Fork fork;                 // side streams of the band smoother's class launches
    ~dm_operator() {
        if (vexec) cudaGraphExecDestroy(vexec);
        if (sexec) cudaGraphExecDestroy(sexec);
        for (int a = 0; a < fork.naux; ++a) {
            cudaStreamDestroy(fork.aux[a]);
            cudaEventDestroy(fork.join[a]);
        }
        if (fork.fork) cudaEventDestroy(fork.fork);
    }
};

namespace {

const GeoLevel& glv(const dm_operator* op, int l) { return *op->geom->lv[l]; }
// Side streams of the band smoother's class launches; none while a trace is
// recording, so that each traced launch is timed alone (as a profiler's
// serialised launch list times it) rather than overlapped with its siblings.
const Fork* fork_of(const dm_operator* op) { return (g_tracer && g_tracer->on) ? nullptr : &op->fork; }
size_t tsize(int prec) { return prec == DM_PREC_F64 ? 8 : (prec == DM_PREC_F32 ? 4 : 2); }

template <typename TC>
BandSchwarz<TC> schwarz_view(const OpLevel& o, const TC* vals) {
    BandSchwarz<TC> b;
    b.off = o.sd_off.get();
    b.copy = o.sd_copy.get();
    b.pos = o.sd_pos.get();
    b.org = o.sd_org.get();
    b.dims = o.sd_dims.get();
    b.vals = vals;
    b.nsub = o.sd_nsub;
    b.ncopies = o.sd_ncopies;
    b.maxrows = o.sd_maxrows;
    b.maxbox = o.sd_maxbox;
    b.fixed = o.sd_fixed;
    for (int k = 0; k < kSchwarzClasses; ++k) {
        b.cls_first[k] = o.sd_cls_first[k];
        b.cls_count[k] = o.sd_cls_count[k];
        b.cls_copies[k] = o.sd_cls_copies[k];
        b.cls_owned[k] = o.sd_cls_owned[k];
    }
    return b;
}

template <typename T, typename TC> struct Pick;
template <> struct Pick<double, double> {
    static const double* A(const GeoLevel& g) { return g.A.get(); }
    static const double* L(const GeoLevel& g) { return g.L.get(); }
    static const double* iV(const GeoLevel& g) { return g.invV.get(); }
    static const double* iD(const OpLevel& o) { return o.invD.get(); }
    static const double* iDs(const OpLevel& o) { return o.invDs.get(); }
    static BandSchwarz<double> bs(const OpLevel& o) { return schwarz_view<double>(o, o.sd_v64.get()); }
};
template <typename T> struct Pick<T, float> {
    static const float* A(const GeoLevel& g) { return g.A32.get(); }
    static const float* L(const GeoLevel& g) { return g.L32.get(); }
    static const float* iV(const GeoLevel& g) { return g.invV32.get(); }
    static const float* iD(const OpLevel& o) { return o.invD32.get(); }
    static const float* iDs(const OpLevel& o) { return o.invDs32.get(); }
    static BandSchwarz<float> bs(const OpLevel& o) { return schwarz_view<float>(o, o.sd_v32.get()); }
};

template <typename T, typename TC>
VecOp<T, TC> vop(const dm_operator* op, int l) {
    const GeoLevel& g = glv(op, l);
    return VecOp<T, TC>{g.g, Pick<T, TC>::A(g), Pick<T, TC>::L(g), Pick<T, TC>::iV(g), Pick<T, TC>::iD(op->ol[l]),
                        op->sigma, l, g.tiles.get(), g.ntiles,
                        op->ol[l].shape ? op->ol[l].stiles.get() : nullptr, op->ol[l].nstiles, op->ol[l].shape};
}
template <typename T, typename TC>
ScalOp<T, TC> sop(const dm_operator* op, int l) {
    const GeoLevel& g = glv(op, l);
    return ScalOp<T, TC>{g.g, Pick<T, TC>::A(g), g.active.get(), Pick<T, TC>::iDs(op->ol[l]), l, g.tiles.get(),
                         g.ntiles};
}

// band smoother sweeps of level l: the fine level, or the coarser ones
int band_sweeps_of(const dm_operator* op, int l) { return l == 0 ? op->mg.band_sweeps : op->mg.band_sweeps_coarse; }

// ---- vector V-cycle: result in rbuf ------------------------------------------------
template <typename T, typename TC>
void vcycle(dm_operator* op, int l, const T* f, T* ebuf, T* rbuf) {
    cudaStream_t s = op->ctx->stream;
    const GeoLevel& g = glv(op, l);
    const size_t vbytes = sizeof(T) * 3 * (size_t)g.g.np;
    if (l == op->nlev - 1) {
        zero(rbuf, vbytes, s);
        dense_coarse_solve<T>(std::is_same<T, double>::value ? op->c_inv.get() : nullptr,
                              std::is_same<T, double>::value ? nullptr : op->c_inv32.get(), op->c_n, op->c_list.get(),
                              nullptr, f, rbuf, op->c_tmp_in.get(), op->c_tmp_out.get(), s);
        return;
    }
    const VecOp<T, TC> o = vop<T, TC>(op, l);
    const double om = op->ol[l].omega;
    double* u = op->band_u.get();
    const int sweeps = band_sweeps_of(op, l);
    const int nu = op->mg.jacobi_sweeps;
    // the iterate and the other work buffer swap roles at every Jacobi sweep
    T* it = ebuf;
    T* tmp = rbuf;
    int k0 = 1;
    if (nu >= 2) {
        // the first sweep from zero, omega D^-1 f, is formed inside the second one
        vec_stencil(o, ST_JACOBI2Z, f, f, tmp, om, s);
        std::swap(it, tmp);
        k0 = 2;
    } else {
        vec_jacobi_zero(o, f, it, om, s);
    }
    for (int k = k0; k < nu; ++k) {
        vec_stencil(o, ST_JACOBI, it, f, tmp, om, s);
        std::swap(it, tmp);
    }
    band_schwarz<T, TC>(Pick<T, TC>::bs(op->ol[l]), o.invD, g.g, g.band.get(), g.nband, f, it, u, om, sweeps, l == 0,
                        s, fork_of(op));
    vec_stencil(o, ST_RESID, it, f, tmp, 0.0, s);
    const GeoLevel& gc = glv(op, l + 1);
    WorkLevel& wc = op->wk[l + 1];
    T* fc = reinterpret_cast<T*>(wc.f.get());
    const bool sym = op->mg.symmetric_transform != 0;
    if (sym) scale_sqrt_a<T, TC>(g.vdom(), Pick<T, TC>::A(g), true, tmp, s);
    face_restrict<T, TC>(g.g, gc.g, Pick<T, TC>::A(gc), tmp, fc, gc.tiles.get(), gc.ntiles, s, sym);
    T* ec = reinterpret_cast<T*>(wc.r.get());
    vcycle<T, TC>(op, l + 1, fc, reinterpret_cast<T*>(wc.e.get()), ec);
    if (sym) scale_sqrt_a<T, TC>(gc.vdom(), Pick<T, TC>::A(gc), false, ec, s);
    face_prolong_add<T, TC>(g.g, gc.g, Pick<T, TC>::A(g), ec, it, g.tiles.get(), g.ntiles, s, sym);
    for (int k = 0; k < nu; ++k) {
        vec_stencil(o, ST_JACOBI, it, f, tmp, om, s);
        std::swap(it, tmp);
    }
    band_schwarz<T, TC>(Pick<T, TC>::bs(op->ol[l]), o.invD, g.g, g.band.get(), g.nband, f, it, u, om, sweeps, l == 0,
                        s, fork_of(op));
    // the cycle's result goes in rbuf
    if (it != rbuf) DM_CUDA(cudaMemcpyAsync(rbuf, it, sizeof(T) * 3 * (size_t)g.g.np, cudaMemcpyDeviceToDevice, s));
}

// ---- scalar V-cycle: result in rbuf -----------------------------------------------
template <typename T, typename TC>
void svcycle(dm_operator* op, int l, const T* f, T* ebuf, T* rbuf) {
    cudaStream_t s = op->ctx->stream;
    const GeoLevel& g = glv(op, l);
    if (l == op->nlev - 1) {
        zero(rbuf, sizeof(T) * (size_t)g.g.np, s);
        dense_coarse_solve<T>(std::is_same<T, double>::value ? op->s_inv.get() : nullptr,
                              std::is_same<T, double>::value ? nullptr : op->s_inv32.get(), op->s_n, op->s_list.get(),
                              op->s_pinned.get(), f, rbuf, op->s_tmp_in.get(), op->s_tmp_out.get(), s);
        return;
    }
    const ScalOp<T, TC> o = sop<T, TC>(op, l);
    const double om = op->ol[l].omega_s;
    scal_jacobi_zero(o, f, ebuf, om, s);
    scal_stencil(o, ST_RESID, ebuf, f, rbuf, 0.0, s);
    const GeoLevel& gc = glv(op, l + 1);
    WorkLevel& wc = op->wk[l + 1];
    T* fc = reinterpret_cast<T*>(wc.sf.get());
    cell_restrict<T>(g.g, gc.g, gc.active.get(), rbuf, fc, gc.tiles.get(), gc.ntiles, s);
    svcycle<T, TC>(op, l + 1, fc, reinterpret_cast<T*>(wc.se.get()), reinterpret_cast<T*>(wc.sr.get()));
    cell_prolong_add<T>(g.g, gc.g, g.active.get(), reinterpret_cast<const T*>(wc.sr.get()), ebuf, g.tiles.get(),
                        g.ntiles, s);
    scal_stencil(o, ST_JACOBI, ebuf, f, rbuf, om, s);
}

// Capture f(...) issued on the context stream into an executable graph.
// Returns false (and leaves *out null) if the capture cannot be made, in which
// case the caller keeps launching kernels directly.
template <class F>
bool capture_graph(dm_operator* op, F&& f, cudaGraphExec_t* out, long long* kernels) {
    cudaStream_t s = op->ctx->stream;
    cudaGraph_t graph = nullptr;
    *out = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const long long before = g_launch_counter ? *g_launch_counter : 0;
    bool ok = true;
    try {
        f();
    } catch (...) {
        ok = false;
    }
    const cudaError_t ec = cudaStreamEndCapture(s, &graph);
    if (!ok || ec != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return false;
    }
    note_allocation();
    const cudaError_t ei = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return false;
    }
    *kernels = (g_launch_counter ? *g_launch_counter : 0) - before;
    if (g_launch_counter) *g_launch_counter = before;   // captured, not executed
    return true;
}

// V-cycles replay as CUDA graphs unless the context traces kernels or the
// environment sets DM_GRAPHS=0 (for profilers that time kernels one launch at
// a time; the same kernels run either way).
bool graphs_allowed(const dm_operator* op) {
    static const bool env_off = [] {
        const char* e = std::getenv("DM_GRAPHS");
        return e && e[0] == '0';
    }();
    return op->graphs && !env_off && !(g_tracer && g_tracer->on);
}

// Learned correction after the V-cycle on the fine level:
//   r = f - (K - sigma A) z,  c = RMS(r) h^2 N(r / RMS(r), A, V),
//   z <- z + alpha c  with alpha = <r, K c> / <K c, K c> (the step along c that
// minimises the residual norm), skipped when alpha <= 0.  So the correction
// never raises the residual of the preconditioned direction.
template <typename T, typename TC>
void learned_correct(dm_operator* op, const T* f, T* z, T* scratch) {
    cudaStream_t s = op->ctx->stream;
    const GeoLevel& g0 = glv(op, 0);
    const VecOp<T, TC> o = vop<T, TC>(op, 0);
    const long long n = 3ll * g0.g.np;
    constexpr int nb = 152 * 2;
    if (op->lc_c.n < sizeof(T) * (size_t)n) {
        op->lc_c.alloc(sizeof(T) * (size_t)n);
        op->lc_kc.alloc(sizeof(T) * (size_t)n);
        op->lc_part.alloc(2 * nb);
        op->lc_host.assign(2 * nb, 0.0);
    }
    T* c = reinterpret_cast<T*>(op->lc_c.get());
    T* kc = reinterpret_cast<T*>(op->lc_kc.get());
    vec_stencil(o, ST_RESID, z, f, scratch, 0.0, s);
    double rr[2];
    dot2<T>(n, scratch, scratch, op->lc_part.get(), op->lc_host.data(), nb, rr, s);
    if (!(rr[0] > 0.0) || op->nopen0 <= 0) return;
    const double scale = std::sqrt(rr[0] / (double)op->nopen0);
    const double h = std::min(g0.g.hx, std::min(g0.g.hy, g0.g.hz));
    LearnedNet& net = *op->lnet;
    net.alloc(g0.g);
    net.features(g0.A.get(), g0.V.get(), 1.0 / scale, scratch, prec_index<T>(), s);
    net.forward(s);
    net.check(s);
    zero(c, sizeof(T) * (size_t)n, s);
    net.add_correction<T>(g0.A.get(), scale * h * h, c, s);
    vec_stencil(o, ST_APPLY, c, (const T*)nullptr, kc, 0.0, s);
    double ab[2];
    dot2<T>(n, scratch, kc, op->lc_part.get(), op->lc_host.data(), nb, ab, s);
    if (ab[1] > 0.0 && ab[0] > 0.0) {
        axpy_store<T>(n, ab[0] / ab[1], c, z, s);
        ++op->learned_applied;
    }
}

// z = M^-1 v on FP64 fine-level vectors: v is converted into the level-0 f
// buffer, the V-cycle runs (as a graph after its first direct run), and the
// result in the level-0 r buffer is converted into z.
// MG input f (storage T) from an FP64 or a float-float vector
template <typename T>
void mg_input(const Domain& D, const double* v, double scale, T* f, cudaStream_t s) {
    DM_REQUIRE(scale == 1.0, DM_ERR_INVALID_ARG, "scaled FP64 preconditioner input");
    convert<T, double>(D, v, f, s);
}
// compact float-float input: scattered into f over the level's list
struct CompactIn {
    const float2* v;
    const int* list;
    long long n;
};
template <typename T>
void mg_input(const Domain& D, const CompactIn& v, double scale, T* f, cudaStream_t s) {
    (void)D;
    ff_scatter<T>(v.n, v.list, scale, v.v, f, s);
}

// z = M^-1 (scale v): one V-cycle (graph-replayed after the first call)
template <typename T, typename TC, typename TIn>
void precond_vec_T(dm_operator* op, const TIn& v, double* z, double scale = 1.0) {
    cudaStream_t s = op->ctx->stream;
    const Domain D = glv(op, 0).vdom();
    WorkLevel& w0 = op->wk[0];
    T* f = reinterpret_cast<T*>(w0.f.get());
    T* e = reinterpret_cast<T*>(w0.e.get());
    T* r = reinterpret_cast<T*>(w0.r.get());
    mg_input<T>(D, v, scale, f, s);
    if (graphs_allowed(op) && op->vcalls > 0) {
        if (!op->vexec && !capture_graph(op, [&] { vcycle<T, TC>(op, 0, f, e, r); }, &op->vexec, &op->vexec_kernels))
            op->graphs = false;
    }
    if (graphs_allowed(op) && op->vexec) {
        DM_CUDA(cudaGraphLaunch(op->vexec, s));
        count_launch(op->vexec_kernels);
    } else {
        vcycle<T, TC>(op, 0, f, e, r);
    }
    ++op->vcalls;
    if (op->lnet && op->learned_active) learned_correct<T, TC>(op, f, r, e);
    convert<double, T>(D, r, z, s);
}

template <typename T, typename TC, typename TIn>
void precond_scal_T(dm_operator* op, const TIn& v, double* z, double scale = 1.0) {
    cudaStream_t s = op->ctx->stream;
    const Domain D = glv(op, 0).sdom();
    WorkLevel& w0 = op->wk[0];
    T* f = reinterpret_cast<T*>(w0.sf.get());
    T* e = reinterpret_cast<T*>(w0.se.get());
    T* r = reinterpret_cast<T*>(w0.sr.get());
    mg_input<T>(D, v, scale, f, s);
    if (graphs_allowed(op) && op->scalls > 0) {
        if (!op->sexec && !capture_graph(op, [&] { svcycle<T, TC>(op, 0, f, e, r); }, &op->sexec, &op->sexec_kernels))
            op->graphs = false;
    }
    if (graphs_allowed(op) && op->sexec) {
        DM_CUDA(cudaGraphLaunch(op->sexec, s));
        count_launch(op->sexec_kernels);
    } else {
        svcycle<T, TC>(op, 0, f, e, r);
    }
    ++op->scalls;
    convert<double, T>(D, r, z, s);
}

template <typename TIn>
void precond_vec(dm_operator* op, const TIn& v, double* z, double scale = 1.0) {
    switch (op->mg.precision) {
        case DM_PREC_F64: precond_vec_T<double, double>(op, v, z, scale); break;
        case DM_PREC_F32: precond_vec_T<float, float>(op, v, z, scale); break;
        default: precond_vec_T<__nv_bfloat16, float>(op, v, z, scale);
    }
}

template <typename TIn>
void precond_scal(dm_operator* op, const TIn& v, double* z, double scale = 1.0) {
    switch (op->mg.precision) {
        case DM_PREC_F64: precond_scal_T<double, double>(op, v, z, scale); break;
        case DM_PREC_F32: precond_scal_T<float, float>(op, v, z, scale); break;
        default: precond_scal_T<__nv_bfloat16, float>(op, v, z, scale);
    }
}

void apply_vec64(dm_operator* op, int l, const double* x, double* y) {
    vec_stencil<double, double>(vop<double, double>(op, l), ST_APPLY, x, nullptr, y, 0.0, op->ctx->stream);
}
void apply_scal64(dm_operator* op, int l, const double* x, double* y) {
    scal_stencil<double, double>(sop<double, double>(op, l), ST_APPLY, x, nullptr, y, 0.0, op->ctx->stream);
}

// sum of x y (times w, nullable) over the fine level's open faces, by the flat
// list kernel once the operator has listed them (over the level's tiles before).
// Callers pass vectors where one factor vanishes on every closed face (the
// operator's output, an A-weighted vector, the solver's own face vectors), so
// the result is the sum over all entries.
double face_dot(dm_context* ctx, const GeoLevel& g0, const double* x, const double* y, const double* w = nullptr) {
    if (g0.nflist >= 0) return dot_list(ctx->red, g0.nflist, g0.flist.get(), x, y, w, ctx->stream);
    const Domain D = g0.vdom();
    double r = 0.0;
    mdot(ctx->red, D, 1, x, D.len(), y, w, &r, ctx->stream);
    return r;
}
double face_norm(dm_context* ctx, const GeoLevel& g0, const double* x, const double* w = nullptr) {
    return std::sqrt(std::max(face_dot(ctx, g0, x, x, w), 0.0));
}

double norm2(dm_context* ctx, const Domain& D, const double* x, const double* w = nullptr) {
    double r = 0.0;
    mdot(ctx->red, D, 1, x, D.len(), x, w, &r, ctx->stream);
    return std::sqrt(std::max(r, 0.0));
}

// Residual of the least-squares problem min |beta e1 - H y| for the first k
// columns of the (k+1) x k Hessenberg H (row stride ld), by Givens QR from
// scratch; y (size k) receives the minimiser.
double hessenberg_lsq(const std::vector<double>& H, int ld, int k, double beta, std::vector<double>* y) {
    std::vector<double> R((size_t)(k + 1) * k), g(k + 1, 0.0);
    for (int i = 0; i <= k; ++i)
        for (int c = 0; c < k; ++c) R[(size_t)i * k + c] = H[(size_t)i * ld + c];
    g[0] = beta;
    for (int c = 0; c < k; ++c) {
        const double a = R[(size_t)c * k + c], b = R[(size_t)(c + 1) * k + c];
        const double r = std::hypot(a, b);
        const double cs = r > 0 ? a / r : 1.0, sn = r > 0 ? b / r : 0.0;
        for (int cc = c; cc < k; ++cc) {
            const double u = R[(size_t)c * k + cc], v = R[(size_t)(c + 1) * k + cc];
            R[(size_t)c * k + cc] = cs * u + sn * v;
            R[(size_t)(c + 1) * k + cc] = -sn * u + cs * v;
        }
        const double gu = g[c], gv = g[c + 1];
        g[c] = cs * gu + sn * gv;
        g[c + 1] = -sn * gu + cs * gv;
    }
    if (y) {
        y->assign(k, 0.0);
        for (int i = k - 1; i >= 0; --i) {
            double acc = g[i];
            for (int c = i + 1; c < k; ++c) acc -= R[(size_t)i * k + c] * (*y)[c];
            (*y)[i] = R[(size_t)i * k + i] != 0.0 ? acc / R[(size_t)i * k + i] : 0.0;
        }
    }
    return std::fabs(g[k]);
}

// Right-preconditioned flexible GMRES (Saad 1993).  The Arnoldi basis is
// orthogonalised by delayed classical Gram-Schmidt (DCGS2, after Swirydowicz,
// Langou, Ananthan, Yang & Thomas 2020): the second Gram-Schmidt pass of each
// basis vector is carried out in the same sweep over the basis as the first
// pass of the next vector, so every iteration reads the basis twice (one
// reduction, one update) instead of four times.  The newest column of H is
// provisional until the next iteration reorthogonalises its vector; the
// residual estimate uses it as it stands (the correction is of rounding
// size), and the end of a cycle confirms with the true FP64 residual.
// x is overwritten.  Returns the iteration count.
struct NoMonitor {
    void operator()(double) const {}
};
// no float-float apply: the iterations apply the FP64 operator and gather
struct NoApplyFF {
    static constexpr bool on = false;
    void operator()(const double*, float2*) const {}
};

// monitor(ratio) is told the residual contraction of every iteration
// The basis lives in the compact index space of `list` (the nl entries of the
// padded domain D that can be nonzero); b, x and the operator work on D.
// apply_ff(z, wf), when ApplyFF::on, forms the operator of an iteration
// straight into the compact float-float vector wf; restart residuals and the
// final check use the FP64 apply.
template <class Apply, class Prec, class Monitor = NoMonitor, class ApplyFF = NoApplyFF>
int fgmres(dm_context* ctx, Fgmres& ws, const Domain& D, const int* list, long long nl, int m, Apply apply, Prec prec,
           const double* b, double* x, double tol, int maxit, double* relres, double abs_tol = 0.0,
           Monitor monitor = Monitor(), ApplyFF apply_ff = ApplyFF()) {
    cudaStream_t s = ctx->stream;
    const long long n = D.len();
    DM_REQUIRE(m >= 1 && 2 * m + 2 < ctx->red.max_cols, DM_ERR_INVALID_ARG, "FGMRES restart length too large");
    DM_REQUIRE(nl >= 1 && nl < (1ll << 31), DM_ERR_INVALID_ARG, "FGMRES: empty basis index space");
    // the compact vectors' length and stride, even for the two-entry passes
    // (the pad entry stays zero: nothing writes it but the update, from zeros)
    const long long nlp = (nl + 1) & ~1ll;
    ws.ensure(n, nlp, m);
    // flat domain of the compact vectors
    Grid3 gc = D.g;
    gc.np = (int)nlp;
    const Domain Dc{gc, nullptr, 0, 1};
    float2* V = ws.V.get();
    float2* wf = ws.wf.get();
    double* Z = ws.Z.get();
    double* w = ws.w.get();
    zero(x, sizeof(double) * n, s);
    // b and every residual vanish outside `list` (closed faces, inactive
    // cells), so their norms run over the list alone
    const double bnorm = std::sqrt(std::max(dot_list(ctx->red, nl, list, b, b, nullptr, s), 0.0));
    if (relres) *relres = 0.0;
    if (bnorm == 0.0) return 0;
    // converged when ||b - A x|| <= thr: relative to ||b||, or the absolute
    // floor abs_tol when the caller knows a better scale than ||b||
    const double thr = std::max(tol * bnorm, abs_tol);
    int total = 0;
    bool first = true;
    double res = 1.0;
    std::vector<double> H((size_t)(m + 1) * m), dots(2 * m + 2), coef(2 * m + 2), y;
    while (total < maxit) {
        // r = b - A x (FP64); V_0 = r / beta in float-float
        double beta = bnorm;
        if (!first) {
            apply(x, w);
            axpby(D, 1.0, b, -1.0, w, s);
            beta = std::sqrt(std::max(dot_list(ctx->red, nl, list, w, w, nullptr, s), 0.0));
        }
        res = beta / bnorm;
        if (beta <= thr) break;
        ff_gather(nl, list, 1.0 / beta, first ? b : w, V, s);
        std::fill(H.begin(), H.end(), 0.0);
        double nu = 1.0;          // norm of the pending vector V_j (provisional)
        double prev = beta;
        int k = 0;                // columns of H built in this cycle
        for (int j = 0; j < m && total < maxit; ++j) {
            float2* Vj = V + (size_t)j * nlp;
            prec(Vj, 1.0 / nu, Z + (size_t)j * n);
            if constexpr (ApplyFF::on) {
                apply_ff(Z + (size_t)j * n, wf);
            } else {
                apply(Z + (size_t)j * n, w);
                ff_gather(nl, list, 1.0, w, wf, s);
            }
            // one sweep: Q^T v, Q^T w, v.v, v.w with Q = V_0 .. V_{j-1} finished
            dcgs_dots(ctx->red, Dc, j, V, nlp, Vj, wf, dots.data(), s);
            double ss = 0.0, sc = 0.0;
            for (int i = 0; i < j; ++i) {
                ss += dots[i] * dots[i];
                sc += dots[i] * dots[j + i];
            }
            const double bj = std::sqrt(std::max(dots[2 * j] - ss, 0.0));
            if (!(bj > 0.0)) break;
            // finish column j-1: its pending vector was Q s + bj V_j
            if (j > 0) {
                for (int i = 0; i < j; ++i) H[(size_t)i * m + (j - 1)] += dots[i];
                H[(size_t)j * m + (j - 1)] = bj;
            }
            // new column: Q^T w and V_j . w for the finished V_j
            const double hj = (dots[2 * j + 1] - sc) / bj;
            for (int i = 0; i < j; ++i) {
                coef[i] = dots[i];
                coef[j + i] = dots[j + i] - hj / bj * dots[i];
                H[(size_t)i * m + j] = dots[j + i];
            }
            H[(size_t)j * m + j] = hj;
            coef[2 * j] = 1.0 / bj;
            coef[2 * j + 1] = hj / bj;
            const double nn2 = dcgs_update(ctx->red, Dc, j, V, nlp, coef.data(), Vj, wf, V + (size_t)(j + 1) * nlp, s);
            nu = std::sqrt(std::max(nn2, 0.0));
            H[(size_t)(j + 1) * m + j] = nu;   // provisional until the next iteration
            k = j + 1;
            ++total;
            const double r = hessenberg_lsq(H, m, k, beta, nullptr);
            if (prev > 0.0) monitor(r / prev);
            prev = r;
            res = r / bnorm;
            if (r <= thr || nu == 0.0) break;
        }
        if (k == 0) break;
        hessenberg_lsq(H, m, k, beta, &y);
        std::vector<double> neg(k);
        for (int i = 0; i < k; ++i) neg[i] = -y[i];
        maxpy(ctx->red, D, k, Z, n, neg.data(), x, s);
        first = false;
        if (res * bnorm <= thr) {
            // confirm with the true residual
            apply(x, w);
            axpby(D, 1.0, b, -1.0, w, s);
            const double tr = std::sqrt(std::max(dot_list(ctx->red, nl, list, w, w, nullptr, s), 0.0)) / bnorm;
            res = tr;
            if (tr * bnorm <= 10.0 * thr) break;
        }
    }
    if (relres) *relres = res;
    return total;
}

// the float-float apply of the projection's scalar iterations (fine level)
struct FFApplyScal {
    static constexpr bool on = true;
    dm_operator* op;
    void operator()(const double* z, float2* wf) const {
        const GeoLevel& l0 = glv(op, 0);
        scal_apply_ff(l0.g, l0.tiles.get(), l0.ntiles, l0.ffA.get(), z, l0.fmapc.get(), wf, op->ctx->stream);
    }
};

// the float-float apply of the shifted solves' iterations (fine level)
struct FFApply {
    static constexpr bool on = true;
    dm_operator* op;
    void operator()(const double* z, float2* wf) const {
        const GeoLevel& l0 = glv(op, 0);
        vec_apply_ff(l0.g, l0.tiles.get(), l0.ntiles, l0.ffA.get(), l0.ffL.get(), l0.ffV.get(), op->sigma, z,
                     l0.fmap.get(), wf, op->ctx->stream);
    }
};

// shifted solves in a row that must switch the learned correction off before
// an operator stops offering it
constexpr int kLearnedStreak = 3;

int solve_vec(dm_operator* op, const double* b, double* x, double tol, int restart, int maxit, double* relres) {
    const Domain n = glv(op, 0).vdom();
    auto apply = [op](const double* in, double* out) { apply_vec64(op, 0, in, out); };
    const GeoLevel& g0 = glv(op, 0);
    const int* fl = g0.flist.get();
    const long long nfl = g0.nflist;
    auto prec = [op, fl, nfl](const float2* in, double scale, double* out) {
        precond_vec(op, CompactIn{in, fl, nfl}, out, scale);
    };
    // the FP64 residual decides on the learned correction: an iteration that
    // contracts by less than 0.8 switches it off for the rest of the solve, and
    // after kLearnedStreak solves in a row that switched it off the operator
    // stops offering it (dm_operator_set_learned offers it again)
    op->learned_active = op->lnet != nullptr && op->learned_streak < kLearnedStreak;
    const bool offered = op->learned_active;
    bool fell_back = false;
    auto monitor = [op, &fell_back](double ratio) {
        if (op->learned_active && ratio > 0.8) {
            op->learned_active = false;
            fell_back = true;
        }
    };
    int it;
    if (op->mg.krylov_ff && g0.ff) {
        it = fgmres(op->ctx, op->vg, n, fl, nfl, restart, apply, prec, b, x, tol, maxit, relres, 0.0, monitor, FFApply{op});
    } else {
        it = fgmres(op->ctx, op->vg, n, fl, nfl, restart, apply, prec, b, x, tol, maxit, relres, 0.0, monitor);
    }
    if (fell_back) {
        ++op->learned_fallbacks;
        ++op->learned_streak;
    } else if (offered) {
        op->learned_streak = 0;
    }
    op->learned_active = false;
    return it;
}

// Iteration cap of the scalar solve inside P_DM, and how many projections of
// one eigensolve may reach it before the solve gives up: a healthy projection
// takes a few tens of iterations, so capped ones mean P_DM is not being
// applied and the eigenpairs cannot be trusted.
constexpr int kProjMaxit = 400;
constexpr int kProjStallLimit = 3;

// y = P_DM x (Eq. proj); x, y padded FP64 fine-level face vectors (may alias)
int project(dm_operator* op, const double* x, double* y, double tol) {
    cudaStream_t s = op->ctx->stream;
    const GeoLevel& g0 = glv(op, 0);
    const Domain nc = g0.sdom();
    double* sv = op->c0.get();
    double* phi = op->c1.get();
    dm_div_a(g0.g, g0.A.get(), x, sv, g0.tiles.get(), g0.ntiles, s);
    // The divergence of a nearly divergence-free x (the shifted solve of a
    // divergence-free vector) is mostly rounding noise, which is not in the
    // range of D A D^T (its component sums are not zero), so a tolerance
    // relative to ||D A x|| cannot be met.  The solve is accurate enough once
    // the residual is tol times the divergence scale of x itself, ||x|| / h.
    const double hmin = std::min(g0.g.hx, std::min(g0.g.hy, g0.g.hz));
    // (D A x sees only the open faces, so they alone set that scale)
    const double xscale = face_norm(op->ctx, g0, x) / hmin;
    auto apply = [op](const double* in, double* out) { apply_scal64(op, 0, in, out); };
    const int* cl = g0.clist.get();
    const long long ncl = g0.nclist;
    auto prec = [op, cl, ncl](const float2* in, double scale, double* out) {
        precond_scal(op, CompactIn{in, cl, ncl}, out, scale);
    };
    double rr = 0.0;
    const int it = (op->mg.krylov_ff && g0.ff)
                       ? fgmres(op->ctx, op->sg, nc, cl, ncl, 40, apply, prec, sv, phi, tol, kProjMaxit, &rr,
                                tol * xscale, NoMonitor(), FFApplyScal{op})
                       : fgmres(op->ctx, op->sg, nc, cl, ncl, 40, apply, prec, sv, phi, tol, kProjMaxit, &rr,
                                tol * xscale);
    dm_sub_grad(g0.g, g0.A.get(), x, phi, y, g0.tiles.get(), g0.ntiles, s);
    return it;
}

// Largest eigenvalue of D^-1 (K - sigma A) on level l by power iteration from
// a seeded random vector on the open faces.  The start is not scaled by D^-1:
// a face or cell with a tiny diagonal would then dominate it, and the
// iteration would report that entry's local eigenvalue (near 1) instead of
// the largest one.
double power_lambda_max(dm_operator* op, int l) {
    cudaStream_t s = op->ctx->stream;
    const GeoLevel& g = glv(op, l);
    const Domain D = g.vdom();
    const long long n = D.len();
    DBuf<double> x(n), y(n);
    fill_random(D, 12345 + l, g.A.get(), x.get(), s);
    double lam = 0.0;
    double nx = norm2(op->ctx, D, x.get());
    if (nx == 0.0) return 1.0;
    scale_copy(D, 1.0 / nx, x.get(), x.get(), s);
    for (int it = 0; it < op->mg.power_iters; ++it) {
        apply_vec64(op, l, x.get(), y.get());
        hadamard(D, op->ol[l].invD.get(), y.get(), y.get(), s);
        const double ny = norm2(op->ctx, D, y.get());
        if (ny == 0.0) break;
        lam = ny;
        scale_copy(D, 1.0 / ny, y.get(), x.get(), s);
    }
    return lam > 0.0 ? lam : 1.0;
}

// Largest eigenvalue of D^-1 D A D^T used for the scalar Jacobi weight.  Every
// row of D A D^T on the active cells sums to zero (a face between an active
// and an inactive cell, or on a conducting outer wall, is closed), or to a
// positive number next to an open magnetic wall (the face to the zero
// potential beyond it), so by Gershgorin the spectrum of D^-1 D A D^T lies in
// [0, 2]; the grid's checkerboard mode comes
// within O(h^2) of 2.  The bound is exact enough and, unlike a power estimate,
// cannot be fooled by a nearly isolated cut cell whose diagonal is ten orders
// of magnitude below the bulk (its local eigenvalue is 1, and an estimate near
// 1 would over-relax the smoother until the scalar cycle diverges).
constexpr double kScalarLambdaMax = 2.0;

void ensure_f32(GeoLevel& g, cudaStream_t s) {
    if (g.A32.get()) return;
    const long long n3 = 3ll * g.g.np, n1 = g.g.np;
    g.A32.alloc(n3);
    g.L32.alloc(n3);
    g.invV32.alloc(n1);
    convert_coeff<float>(n3, g.A.get(), g.A32.get(), s);
    convert_coeff<float>(n3, g.L.get(), g.L32.get(), s);
    convert_coeff<float>(n1, g.invV.get(), g.invV32.get(), s);
}

__global__ void k_invert_diag(long long n, const double* __restrict__ d, double* __restrict__ inv) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        inv[r] = d[r] != 0.0 ? 1.0 / d[r] : 0.0;
}
void invert_diag(long long n, const double* d, double* inv, cudaStream_t s) {
    const int b = (int)std::min<long long>((n + 255) / 256, 152 * 8);
    launch("k_invert_diag", k_invert_diag, b, 256, 0, s, n, d, inv);
}

// Time the tiled Jacobi stencil of `level` for every tile shape and keep the
// fastest (CUDA events on the context stream; 2 warm-up + 5 timed launches on
// the level's work buffers).  Choices are cached in the context.
template <typename T, typename TC>
void autotune_level(dm_operator* op, int l) {
    cudaStream_t s = op->ctx->stream;
    GeoLevel& g = *const_cast<dm_geometry*>(op->geom)->lv[l];
    OpLevel& o = op->ol[l];
    const std::array<int, 4> key{g.g.nx, g.g.ny, g.g.nz, op->mg.precision};
    for (const auto& kv : op->ctx->tuned)
        if (kv.first == key) {
            o.shape = kv.second;
            break;
        }
    std::vector<DBuf<int>> lists(kStencilShapes);
    std::vector<int> counts(kStencilShapes, 0);
    DBuf<int> cnt(1);
    for (int sh = 1; sh < kStencilShapes; ++sh) {
        int sy, sz;
        stencil_shape_dims(sh, sy, sz);
        const int nt = ((g.g.nx + TX) / TX) * ((g.g.ny + sy) / sy) * ((g.g.nz + sz) / sz);
        DBuf<int> flags(nt);
        lists[sh].alloc(nt);
        counts[sh] = geom_tiles_shape(g.g, sy, sz, g.A.get(), g.active.get(), lists[sh].get(), flags.get(), cnt.get(), s);
    }
    bool cached = false;
    for (const auto& kv : op->ctx->tuned) cached |= kv.first == key;
    if (!cached) {
        WorkLevel& w = op->wk[l];
        const T* x = reinterpret_cast<const T*>(w.e.get());
        const T* f = reinterpret_cast<const T*>(w.f.get());
        T* y = reinterpret_cast<T*>(w.r.get());
        cudaEvent_t e0, e1;
        note_allocation();
        DM_CUDA(cudaEventCreate(&e0));
        note_allocation();
        DM_CUDA(cudaEventCreate(&e1));
        float best = 1e30f;
        int best_shape = 0;
        for (int sh = 0; sh < kStencilShapes; ++sh) {
            o.shape = sh;
            o.nstiles = counts[sh];
            VecOp<T, TC> vo = vop<T, TC>(op, l);
            if (sh) vo.stiles = lists[sh].get();
            for (int r = 0; r < 2; ++r) vec_stencil(vo, ST_JACOBI, x, f, y, 0.5, s);
            DM_CUDA(cudaEventRecord(e0, s));
            for (int r = 0; r < 5; ++r) vec_stencil(vo, ST_JACOBI, x, f, y, 0.5, s);
            DM_CUDA(cudaEventRecord(e1, s));
            DM_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            DM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                best_shape = sh;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        o.shape = best_shape;
        op->ctx->tuned.push_back({key, o.shape});
    }
    o.nstiles = counts[o.shape];
    if (o.shape) o.stiles = std::move(lists[o.shape]);
    zero(op->wk[l].r.get(), op->wk[l].r.n, s);
}

// Use tile shape `sh` for the vector stencil of level l.
void set_level_shape(dm_operator* op, int l, int sh) {
    GeoLevel& g = *const_cast<dm_geometry*>(op->geom)->lv[l];
    OpLevel& o = op->ol[l];
    o.shape = sh;
    o.nstiles = 0;
    o.stiles = DBuf<int>();
    if (sh == 0) return;
    int sy, sz;
    stencil_shape_dims(sh, sy, sz);
    const int nt = ((g.g.nx + TX) / TX) * ((g.g.ny + sy) / sy) * ((g.g.nz + sz) / sz);
    DBuf<int> flags(nt), cnt(1);
    o.stiles.alloc(nt);
    o.nstiles = geom_tiles_shape(g.g, sy, sz, g.A.get(), g.active.get(), o.stiles.get(), flags.get(), cnt.get(),
                                 op->ctx->stream);
}

void setup_operator(dm_operator* op) {
    cudaStream_t s = op->ctx->stream;
    dm_geometry* geom = const_cast<dm_geometry*>(op->geom);
    // levels used by this operator
    int nl = 1;
    while (nl < (int)geom->lv.size()) {
        const Grid3& g = geom->lv[nl - 1]->g;
        if (!can_coarsen(g.nx, g.ny, g.nz, op->mg.max_coarse)) break;
        // a level this small is solved densely instead: its coarse-level
        // launches would be latency-bound for no gain
        if (op->mg.dense_coarse > 0 && geom->lv[nl - 1]->nopen <= op->mg.dense_coarse) break;
        ++nl;
    }
    op->nlev = nl;
    op->ol.resize(nl);
    op->wk.resize(nl);
    const bool lowp = op->mg.precision != DM_PREC_F64;
    const size_t ts = tsize(op->mg.precision);
    int max_band = 1;
    for (int l = 0; l < nl; ++l) {
        GeoLevel& g = *geom->lv[l];
        if (lowp) {
            std::lock_guard<std::mutex> lock(geom->mu);
            ensure_f32(g, s);
            Sync::stream(s);
        }
        OpLevel& o = op->ol[l];
        const long long n3 = 3ll * g.g.np, n1 = g.g.np;
        DBuf<double> d(n3);
        vec_diagonal(g.g, g.A.get(), g.L.get(), g.invV.get(), op->sigma, d.get(), s);
        o.invD.alloc(n3);
        invert_diag(n3, d.get(), o.invD.get(), s);
        DBuf<double> ds(n1);
        scal_diagonal(g.g, g.A.get(), g.active.get(), ds.get(), s);
        o.invDs.alloc(n1);
        invert_diag(n1, ds.get(), o.invDs.get(), s);
        if (lowp) {
            o.invD32.alloc(n3);
            o.invDs32.alloc(n1);
            convert_coeff<float>(n3, o.invD.get(), o.invD32.get(), s);
            convert_coeff<float>(n1, o.invDs.get(), o.invDs32.get(), s);
        }
        if (g.nband > 0 && l + 1 < nl) {
            SchwarzLayout sl;
            band_schwarz_setup(g.g, g.band.get(), g.nband, op->mg.band_brick, sl, s);
            o.sd_nsub = (int)sl.off.size() - 1;
            o.sd_ncopies = (int)sl.copy.size();
            o.sd_maxrows = sl.maxrows;
            o.sd_maxbox = sl.maxbox;
            o.sd_fixed = sl.fixed;
            for (int k = 0; k < kSchwarzClasses; ++k) {
                o.sd_cls_first[k] = sl.cls_first[k];
                o.sd_cls_count[k] = sl.cls_count[k];
                o.sd_cls_copies[k] = sl.cls_copies[k];
                o.sd_cls_owned[k] = sl.cls_owned[k];
            }
            switch (op->mg.precision) {
                case DM_PREC_F64: band_schwarz_prepare<double, double>(sl); break;
                case DM_PREC_F32: band_schwarz_prepare<float, float>(sl); break;
                default: band_schwarz_prepare<__nv_bfloat16, float>(sl);
            }
            auto upload = [&](DBuf<int>& d, const std::vector<int>& h) {
                d.alloc(h.size(), false);
                DM_CUDA(cudaMemcpyAsync(d.get(), h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice, s));
            };
            upload(o.sd_off, sl.off);
            upload(o.sd_copy, sl.copy);
            upload(o.sd_pos, sl.pos);
            upload(o.sd_org, sl.org);
            upload(o.sd_dims, sl.dims);
            const size_t nb = (size_t)g.nband, nv = (size_t)kBandSlots * o.sd_ncopies;
            DBuf<double> rows(kBandSlots * nb, false);
            band_slots(g.g, g.A.get(), g.L.get(), g.invV.get(), op->sigma, g.band.get(), g.nband, rows.get(), s);
            o.sd_v64.alloc(nv, false);
            band_copy_vals(o.sd_copy.get(), o.sd_ncopies, rows.get(), g.nband, o.sd_v64.get(), s);
            if (lowp) {
                o.sd_v32.alloc(nv, false);
                convert_coeff<float>((long long)nv, o.sd_v64.get(), o.sd_v32.get(), s);
            }
            Sync::stream(s);   // the host layout and the row buffer are released on return
        }
        WorkLevel& w = op->wk[l];
        w.f.alloc(ts * n3);
        w.e.alloc(ts * n3);
        w.r.alloc(ts * n3);
        w.sf.alloc(ts * n1);
        w.se.alloc(ts * n1);
        w.sr.alloc(ts * n1);
        max_band = std::max(max_band, g.nband);
    }
    op->band_u.alloc((size_t)max_band);
    {
        note_allocation();
        DM_CUDA(cudaEventCreateWithFlags(&op->fork.fork, cudaEventDisableTiming));
        for (int a = 0; a < kForkStreams; ++a) {
            note_allocation();
            DM_CUDA(cudaStreamCreateWithFlags(&op->fork.aux[a], cudaStreamNonBlocking));
            note_allocation();
            DM_CUDA(cudaEventCreateWithFlags(&op->fork.join[a], cudaEventDisableTiming));
            op->fork.naux = a + 1;
        }
    }
    {
        // compact index spaces of the fine level's Krylov bases
        GeoLevel& g0 = *const_cast<dm_geometry*>(geom)->lv[0];
        std::lock_guard<std::mutex> lock(const_cast<dm_geometry*>(geom)->mu);
        if (g0.nflist < 0) {
            g0.nflist = list_flagged<double>(3ll * g0.g.np, g0.A.get(), g0.flist, s);
            g0.nclist = list_flagged<unsigned char>((long long)g0.g.np, g0.active.get(), g0.clist, s);
        }
        if (op->mg.krylov_ff && !g0.ff) {
            const long long n3 = 3ll * g0.g.np;
            g0.ffA = DBuf<float2>(n3);
            g0.ffL = DBuf<float2>(n3);
            g0.ffV = DBuf<float2>(g0.g.np);
            g0.fmap = DBuf<int>(n3);
            note_allocation();
            to_ff(n3, g0.A.get(), g0.ffA.get(), s);
            to_ff(n3, g0.L.get(), g0.ffL.get(), s);
            to_ff(g0.g.np, g0.invV.get(), g0.ffV.get(), s);
            compact_map(n3, g0.flist.get(), g0.nflist, g0.fmap.get(), s);
            g0.fmapc = DBuf<int>(g0.g.np);
            compact_map(g0.g.np, g0.clist.get(), g0.nclist, g0.fmapc.get(), s);
            Sync::stream(s);
            g0.ff = true;
        }
    }
    if (op->mg.stencil_shape >= 0) {
        for (int l = 0; l + 1 < nl; ++l) set_level_shape(op, l, op->mg.stencil_shape);
    } else if (op->mg.autotune) {
        for (int l = 0; l + 1 < nl; ++l) {
            switch (op->mg.precision) {
                case DM_PREC_F64: autotune_level<double, double>(op, l); break;
                case DM_PREC_F32: autotune_level<float, float>(op, l); break;
                default: autotune_level<__nv_bfloat16, float>(op, l);
            }
        }
    }
    {
        DBuf<int> cnt(1);
        long long tot = 0, fine = 0;
        for (int l = 0; l < nl; ++l) {
            const GeoLevel& g = *geom->lv[l];
            const long long c = count_positive(3ll * g.g.np, g.A.get(), cnt.get(), s);
            if (l == 0) fine = c;
            tot += c;
        }
        op->complexity = fine > 0 ? (double)tot / (double)fine : 1.0;
        op->nopen0 = fine;
    }
    // Jacobi weights from the largest eigenvalue of D^-1 (K - sigma A) and of
    // D^-1 D A D^T
    for (int l = 0; l + 1 < nl; ++l) {
        op->ol[l].omega = op->mg.omega_scale / power_lambda_max(op, l);
        op->ol[l].omega_s = op->mg.omega_scale / kScalarLambdaMax;
    }
    // coarsest vector level: dense inverse over the open faces
    {
        GeoLevel& g = *geom->lv[nl - 1];
        DBuf<int> cnt(1);
        op->c_list.alloc(3ll * g.g.np);
        op->c_n = geom_open_faces(g.g, g.A.get(), op->c_list.get(), cnt.get(), s);
        const int n = op->c_n;
        DM_REQUIRE(n > 0, DM_ERR_GEOMETRY, "coarsest level has no open face");
        DM_REQUIRE(n <= 6000, DM_ERR_INVALID_ARG, "coarsest level too large for the dense solve; raise max_coarse");
        op->c_inv.alloc((size_t)n * n);
        vec_dense_assemble(g.g, g.A.get(), g.L.get(), g.invV.get(), op->sigma, op->c_list.get(), n, op->c_inv.get(), s);
        DBuf<double> work(2ull * n * n + n);
        DBuf<int> flag(1);
        DM_REQUIRE(dense_inverse(op->c_inv.get(), n, work.get(), flag.get(), s), DM_ERR_NO_CONVERGENCE,
                   "coarsest K - sigma A is singular (sigma is an eigenvalue of the coarsest grid)");
        if (lowp) {
            op->c_inv32.alloc((size_t)n * n);
            convert_coeff<float>((long long)n * n, op->c_inv.get(), op->c_inv32.get(), s);
        }
        op->c_tmp_in.alloc(n);
        op->c_tmp_out.alloc(n);
    }
    // coarsest scalar level: dense inverse with one pinned cell per component
    {
        GeoLevel& g = *geom->lv[nl - 1];
        DBuf<int> cnt(1);
        op->s_list.alloc(g.g.np);
        DBuf<unsigned char> act(g.g.np);
        op->s_n = geom_active_cells(g.g, g.A.get(), op->s_list.get(), act.get(), cnt.get(), s);
        const int n = op->s_n;
        DM_REQUIRE(n > 0, DM_ERR_GEOMETRY, "coarsest level has no active cell");
        DBuf<int> label(n);
        op->s_pinned.alloc(n);
        cell_components_pin(g.g, g.A.get(), op->s_list.get(), n, label.get(), op->s_pinned.get(), s);
        op->s_inv.alloc((size_t)n * n);
        scal_dense_assemble(g.g, g.A.get(), op->s_list.get(), op->s_pinned.get(), n, op->s_inv.get(), s);
        DBuf<double> work(2ull * n * n + n);
        DBuf<int> flag(1);
        DM_REQUIRE(dense_inverse(op->s_inv.get(), n, work.get(), flag.get(), s), DM_ERR_NO_CONVERGENCE,
                   "coarsest scalar Laplacian is singular after pinning");
        if (lowp) {
            op->s_inv32.alloc((size_t)n * n);
            convert_coeff<float>((long long)n * n, op->s_inv.get(), op->s_inv32.get(), s);
        }
        op->s_tmp_in.alloc(n);
        op->s_tmp_out.alloc(n);
    }
    const long long n3 = 3ll * glv(op, 0).g.np, n1 = glv(op, 0).g.np;
    op->t0.alloc(n3);
    op->t1.alloc(n3);
    op->t2.alloc(n3);
    op->t3.alloc(n3);
    op->c0.alloc(n1);
    op->c1.alloc(n1);
    Sync::stream(s);
}

// natural <-> padded staging helpers (host or device caller buffers)
void stage_in(dm_context* ctx, const double* src, int on_device, size_t count, DBuf<double>& tmp, const double** dev) {
    if (on_device) {
        *dev = src;
        return;
    }
    tmp.alloc(count, false);
    DM_CUDA(cudaMemcpyAsync(tmp.get(), src, sizeof(double) * count, cudaMemcpyHostToDevice, ctx->stream));
    *dev = tmp.get();
}
void stage_out(dm_context* ctx, const double* dev, double* dst, int on_device, size_t count) {
    DM_CUDA(cudaMemcpyAsync(dst, dev, sizeof(double) * count,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    DM_CUDA(cudaStreamSynchronize(ctx->stream));
}

__global__ void k_mask_open(long long n, const double* __restrict__ A, double* __restrict__ x) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        if (!(A[r] > 0.0)) x[r] = 0.0;
}

// caller face vector -> padded level-l vector; entries on closed faces are
// dropped (closed faces always hold 0)
void faces_in(dm_operator* op, int l, const double* nat, int on_device, double* pad) {
    const GeoLevel& gl = glv(op, l);
    const Grid3& g = gl.g;
    DBuf<double> tmp;
    const double* d = nullptr;
    stage_in(op->ctx, nat, on_device, (size_t)natural_faces(g), tmp, &d);
    zero(pad, sizeof(double) * 3 * (size_t)g.np, op->ctx->stream);
    pack_faces(g, d, pad, op->ctx->stream);
    const long long n3 = 3ll * g.np;
    launch("k_mask_open", k_mask_open, (int)std::min<long long>((n3 + 255) / 256, 1216), 256, 0, op->ctx->stream, n3,
           gl.A.get(), pad);
    Sync::stream(op->ctx->stream);
}
void faces_out(dm_operator* op, int l, const double* pad, double* nat, int on_device) {
    const Grid3& g = glv(op, l).g;
    const size_t nf = (size_t)natural_faces(g);
    if (on_device) {
        unpack_faces(g, pad, nat, op->ctx->stream);
        Sync::stream(op->ctx->stream);
    } else {
        DBuf<double> tmp(nf, false);
        unpack_faces(g, pad, tmp.get(), op->ctx->stream);
        stage_out(op->ctx, tmp.get(), nat, 0, nf);
    }
}
void cells_in(dm_operator* op, int l, const double* nat, int on_device, double* pad) {
    const Grid3& g = glv(op, l).g;
    DBuf<double> tmp;
    const double* d = nullptr;
    stage_in(op->ctx, nat, on_device, (size_t)natural_cells(g), tmp, &d);
    zero(pad, sizeof(double) * (size_t)g.np, op->ctx->stream);
    pack_cells(g, d, pad, op->ctx->stream);
    Sync::stream(op->ctx->stream);
}
void cells_out(dm_operator* op, int l, const double* pad, double* nat, int on_device) {
    const Grid3& g = glv(op, l).g;
    const size_t nc = (size_t)natural_cells(g);
    if (on_device) {
        unpack_cells(g, pad, nat, op->ctx->stream);
        Sync::stream(op->ctx->stream);
    } else {
        DBuf<double> tmp(nc, false);
        unpack_cells(g, pad, tmp.get(), op->ctx->stream);
        stage_out(op->ctx, tmp.get(), nat, 0, nc);
    }
}

// run f(T**) on copies of level-l FP64 face vectors converted to storage type T
template <typename T, class F>
void with_mg_vectors(dm_operator* op, int l, int count, double* const* pads, F&& f) {
    cudaStream_t s = op->ctx->stream;
    const Domain D = glv(op, l).vdom();
    const long long n = D.len();
    std::vector<DBuf<T>> b(count);
    std::vector<T*> p(count);
    for (int i = 0; i < count; ++i) {
        b[i].alloc(n);
        p[i] = b[i].get();
        convert<T, double>(D, pads[i], p[i], s);
    }
    f(p.data());
    for (int i = 0; i < count; ++i) convert<double, T>(D, p[i], pads[i], s);
    Sync::stream(s);
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

dm_status dm_context_create(int device, void* cuda_stream, dm_context** out) {
    if (!out) return DM_ERR_INVALID_ARG;
    *out = nullptr;
    auto* ctx = new (std::nothrow) dm_context();
    if (!ctx) return DM_ERR_OOM;
    const dm_status st = guarded(ctx, [&] {
        int ndev = 0;
        DM_CUDA(cudaGetDeviceCount(&ndev));
        DM_REQUIRE(device >= 0 && device < ndev, DM_ERR_INVALID_ARG, "no such CUDA device");
        DM_CUDA(cudaSetDevice(device));
        ctx->device = device;
        if (cuda_stream) {
            ctx->stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            // a blocking stream: ordered after work the caller queued on the
            // legacy default stream (e.g. torch copies of input tensors)
            note_allocation();
            DM_CUDA(cudaStreamCreate(&ctx->stream));
            ctx->own_stream = true;
        }
        reducer_init(ctx->red, 160);
    });
    if (st != DM_OK) {
        delete ctx;
        return st;
    }
    *out = ctx;
    return DM_OK;
}

void dm_context_destroy(dm_context* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    reducer_free(ctx->red);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char* dm_last_error(const dm_context* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

dm_status dm_trace_enable(dm_context* ctx, int on) {
    if (!ctx) return DM_ERR_INVALID_ARG;
    return guarded(ctx, [&] {
        if (on) ctx->tracer.reset();
        else ctx->tracer.resolve();
        ctx->tracer.on = on != 0;
    });
}

int dm_trace_count(dm_context* ctx) {
    if (!ctx) return 0;
    if (guarded(ctx, [&] { ctx->tracer.resolve(); }) != DM_OK) return 0;
    return (int)ctx->tracer.stats.size();
}

dm_status dm_trace_entry(dm_context* ctx, int i, char* name, int name_cap, long long* launches, double* total_ms) {
    if (!ctx || i < 0) return DM_ERR_INVALID_ARG;
    return guarded(ctx, [&] {
        ctx->tracer.resolve();
        DM_REQUIRE(i < (int)ctx->tracer.stats.size(), DM_ERR_INVALID_ARG, "trace entry out of range");
        const Tracer::Stat& st = ctx->tracer.stats[i];
        if (name && name_cap > 0) {
            std::strncpy(name, st.name.c_str(), (size_t)name_cap - 1);
            name[name_cap - 1] = 0;
        }
        if (launches) *launches = st.launches;
        if (total_ms) *total_ms = st.ms;
    });
}
long long dm_context_launch_count(const dm_context* ctx) { return ctx ? ctx->launches : 0; }

dm_status dm_measure_fma_rates(dm_context* ctx, double* fp64_tflops, double* fp32_tflops) {
    if (!ctx) return DM_ERR_INVALID_ARG;
    return guarded(ctx, [&] {
        DM_CUDA(cudaSetDevice(ctx->device));
        double r64 = 0.0, r32 = 0.0;
        probe_fma_rates(ctx->stream, &r64, &r32);
        if (fp64_tflops) *fp64_tflops = r64 * 1e-12;
        if (fp32_tflops) *fp32_tflops = r32 * 1e-12;
    });
}

dm_status dm_trace_entry_bytes(dm_context* ctx, int i, double* bytes) {
    if (!ctx || i < 0 || !bytes) return DM_ERR_INVALID_ARG;
    return guarded(ctx, [&] {
        ctx->tracer.resolve();
        DM_REQUIRE(i < (int)ctx->tracer.stats.size(), DM_ERR_INVALID_ARG, "trace entry out of range");
        *bytes = ctx->tracer.stats[i].bytes;
    });
}

long long dm_debug_allocation_count(void) { return g_allocations.load(std::memory_order_relaxed); }

}  // extern "C"

namespace {

// The multigrid levels of a geometry: `fine` fills level 0's L, A and V
// (padded layouts); every coarser level averages the level above.
template <class Fine>
dm_status build_geometry(dm_context* ctx, int nx, int ny, int nz, double dx, double dy, double dz, Fine&& fine,
                         dm_geometry** out) {
    *out = nullptr;
    auto geom = std::make_unique<dm_geometry>();
    const dm_status st = guarded(ctx, [&] {
        DM_REQUIRE(nx >= 2 && ny >= 2 && nz >= 2, DM_ERR_INVALID_ARG, "grid needs at least 2 cells per dimension");
        DM_REQUIRE(dx > 0 && dy > 0 && dz > 0, DM_ERR_INVALID_ARG, "cell sizes must be positive");
        DM_CUDA(cudaSetDevice(ctx->device));
        cudaStream_t s = ctx->stream;
        geom->ctx = ctx;
        int cx = nx, cy = ny, cz = nz;
        double hx = dx, hy = dy, hz = dz;
        for (int l = 0;; ++l) {
            auto lv = std::make_unique<GeoLevel>();
            lv->g = make_grid(cx, cy, cz, hx, hy, hz);
            const long long n3 = 3ll * lv->g.np, n1 = lv->g.np;
            lv->A.alloc(n3);
            lv->L.alloc(n3);
            lv->V.alloc(n1);
            lv->invV.alloc(n1);
            if (l == 0) {
                fine(*lv, s);
                Sync::stream(s);
            } else {
                const GeoLevel& f = *geom->lv[l - 1];
                geom_coarsen(f.g, lv->g, f.L.get(), f.A.get(), f.V.get(), lv->L.get(), lv->A.get(), lv->V.get(), s);
            }
            geom_inv_volume(lv->g, lv->V.get(), lv->invV.get(), s);
            // smoother band and active cells
            DBuf<int> flag(n1), cnt(1);
            lv->band.alloc(n3);
            lv->nband = geom_band(lv->g, lv->A.get(), lv->V.get(), flag.get(), lv->band.get(), cnt.get(), s);
            lv->active.alloc(n1);
            geom_active_cells(lv->g, lv->A.get(), nullptr, lv->active.get(), cnt.get(), s);
            {
                const int nt = tiles_x(lv->g) * tiles_y(lv->g) * tiles_z(lv->g);
                DBuf<int> tflags(nt);
                lv->tiles.alloc(nt);
                lv->ntiles = geom_tiles(lv->g, lv->A.get(), lv->active.get(), lv->tiles.get(), tflags.get(), cnt.get(), s);
            }
            lv->nopen = count_positive(n3, lv->A.get(), cnt.get(), s);
            lv->g.nopen = lv->nopen;
            lv->g.nact = count_flags(n1, lv->active.get(), cnt.get(), s);
            geom->lv.push_back(std::move(lv));
            if (!can_coarsen(cx, cy, cz, 4)) break;
            cx /= 2; cy /= 2; cz /= 2;
            hx *= 2; hy *= 2; hz *= 2;
        }
        Sync::stream(s);
    });
    if (st != DM_OK) return st;
    *out = geom.release();
    return DM_OK;
}

}  // namespace

extern "C" {

dm_status dm_geometry_create(dm_context* ctx, int nx, int ny, int nz, double dx, double dy, double dz,
                             const double origin[3], const double* phi, int phi_on_device, double a_min,
                             dm_geometry** out) {
    return dm_geometry_create_walls(ctx, nx, ny, nz, dx, dy, dz, origin, phi, phi_on_device, a_min, nullptr, out);
}

dm_status dm_geometry_create_walls(dm_context* ctx, int nx, int ny, int nz, double dx, double dy, double dz,
                                   const double origin[3], const double* phi, int phi_on_device, double a_min,
                                   const int walls[6], dm_geometry** out) {
    if (!ctx || !out || !phi) return DM_ERR_INVALID_ARG;
    *out = nullptr;
    (void)origin;
    if (!(a_min >= 0.0 && a_min < 1.0)) {
        ctx->err = "a_min must be in [0, 1)";
        return DM_ERR_INVALID_ARG;
    }
    int pmc = 0;
    for (int w = 0; walls && w < 6; ++w) {
        if (walls[w] != DM_WALL_PEC && walls[w] != DM_WALL_PMC) {
            ctx->err = "walls[" + std::to_string(w) + "] is neither DM_WALL_PEC nor DM_WALL_PMC";
            return DM_ERR_INVALID_ARG;
        }
        if (walls[w] == DM_WALL_PMC) pmc |= 1 << w;
    }
    return build_geometry(ctx, nx, ny, nz, dx, dy, dz, [&](GeoLevel& lv, cudaStream_t s) {
        DBuf<double> phi_pad(lv.g.np);
        const size_t nn = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
        DBuf<double> tmp;
        const double* dphi = nullptr;
        stage_in(ctx, phi, phi_on_device, nn, tmp, &dphi);
        {
            DBuf<int> bad(1);
            const int nbad = count_nonfinite((long long)nn, dphi, bad.get(), s);
            DM_REQUIRE(nbad == 0, DM_ERR_GEOMETRY,
                       "level set: " + std::to_string(nbad) + " of " + std::to_string(nn) +
                           " node values are NaN or infinite");
        }
        pack_nodes(lv.g, dphi, phi_pad.get(), s);
        geom_fractions(lv.g, phi_pad.get(), pmc, lv.L.get(), lv.A.get(), lv.V.get(), s);
        if (a_min > 0.0) geom_neglect_faces(lv.g, a_min, lv.L.get(), lv.A.get(), s);
        Sync::stream(s);
    }, out);
}

dm_status dm_geometry_create_from_fractions(dm_context* ctx, int nx, int ny, int nz, double dx, double dy, double dz,
                                            const double* L, const double* A, const double* V, int on_device,
                                            dm_geometry** out) {
    if (!ctx || !out || !L || !A || !V) return DM_ERR_INVALID_ARG;
    *out = nullptr;
    return build_geometry(ctx, nx, ny, nz, dx, dy, dz, [&](GeoLevel& lv, cudaStream_t s) {
        const Grid3& g = lv.g;
        const size_t ne = (size_t)natural_edges(g), nf = (size_t)natural_faces(g), nc = (size_t)natural_cells(g);
        DBuf<double> tl, ta, tv;
        const double *dl = nullptr, *da = nullptr, *dv = nullptr;
        stage_in(ctx, L, on_device, ne, tl, &dl);
        stage_in(ctx, A, on_device, nf, ta, &da);
        stage_in(ctx, V, on_device, nc, tv, &dv);
        DBuf<int> bad(1);
        const int bl = count_outside((long long)ne, dl, 0.0, 1.0, bad.get(), s);
        const int ba = count_outside((long long)nf, da, 0.0, 1.0, bad.get(), s);
        const int bv = count_outside((long long)nc, dv, 0.0, std::numeric_limits<double>::max(), bad.get(), s);
        DM_REQUIRE(bl == 0 && ba == 0 && bv == 0, DM_ERR_GEOMETRY,
                   "fractions: " + std::to_string(bl) + " edge and " + std::to_string(ba) +
                       " face values outside [0, 1], " + std::to_string(bv) + " cell values negative or not finite");
        pack_edges(g, dl, lv.L.get(), s);
        pack_faces(g, da, lv.A.get(), s);
        pack_cells(g, dv, lv.V.get(), s);
        geom_close_walls(g, lv.L.get(), lv.A.get(), s);
        Sync::stream(s);
    }, out);
}

void dm_geometry_destroy(dm_geometry* geom) {
    if (!geom) return;
    if (geom->ctx) cudaStreamSynchronize(geom->ctx->stream);
    delete geom;
}

int dm_geometry_num_levels(const dm_geometry* geom) { return geom ? (int)geom->lv.size() : 0; }

dm_status dm_geometry_level_info(const dm_geometry* geom, int level, int dims[3], long long counts[4]) {
    if (!geom || level < 0 || level >= (int)geom->lv.size()) return DM_ERR_INVALID_ARG;
    return guarded(geom->ctx, [&] {
        const GeoLevel& g = *geom->lv[level];
        if (dims) { dims[0] = g.g.nx; dims[1] = g.g.ny; dims[2] = g.g.nz; }
        if (counts) {
            counts[0] = natural_faces(g.g);
            counts[1] = natural_edges(g.g);
            counts[2] = natural_cells(g.g);
            counts[3] = g.nopen;
        }
    });
}

dm_status dm_geometry_fractions(const dm_geometry* geom, int level, double* L, double* A, double* V, int on_device) {
    if (!geom || level < 0 || level >= (int)geom->lv.size()) return DM_ERR_INVALID_ARG;
    return guarded(geom->ctx, [&] {
        const GeoLevel& g = *geom->lv[level];
        cudaStream_t s = geom->ctx->stream;
        auto out = [&](auto unpack, const double* pad, double* dst, size_t count) {
            if (!dst) return;
            if (on_device) {
                unpack(g.g, pad, dst, s);
                Sync::stream(s);
            } else {
                DBuf<double> tmp(count, false);
                unpack(g.g, pad, tmp.get(), s);
                stage_out(geom->ctx, tmp.get(), dst, 0, count);
            }
        };
        out(unpack_edges, g.L.get(), L, (size_t)natural_edges(g.g));
        out(unpack_faces, g.A.get(), A, (size_t)natural_faces(g.g));
        out(unpack_cells, g.V.get(), V, (size_t)natural_cells(g.g));
    });
}

void dm_mg_params_default(dm_mg_params* p) {
    if (!p) return;
    p->max_coarse = 4;
    p->band_sweeps = 24;
    p->band_brick = 8;
    p->omega_scale = 1.7;
    p->power_iters = 30;
    p->precision = DM_PREC_F64;
    p->autotune = 1;
    p->stencil_shape = -1;
    p->band_sweeps_coarse = 16;
    p->symmetric_transform = 0;
    p->dense_coarse = 2048;
    p->krylov_ff = 1;
    p->jacobi_sweeps = 2;
}

dm_status dm_operator_create(dm_context* ctx, const dm_geometry* geom, double sigma, const dm_mg_params* mg,
                             dm_operator** out) {
    if (!ctx || !geom || !out) return DM_ERR_INVALID_ARG;
    *out = nullptr;
    auto op = std::make_unique<dm_operator>();
    const dm_status st = guarded(ctx, [&] {
        DM_CUDA(cudaSetDevice(ctx->device));
        op->ctx = ctx;
        op->geom = geom;
        op->sigma = sigma;
        dm_mg_params_default(&op->mg);
        if (mg) op->mg = *mg;
        DM_REQUIRE(op->mg.max_coarse >= 4, DM_ERR_INVALID_ARG, "max_coarse must be >= 4");
        DM_REQUIRE(op->mg.dense_coarse >= 0 && op->mg.dense_coarse <= 6000, DM_ERR_INVALID_ARG,
                   "dense_coarse must be in [0, 6000]");
        DM_REQUIRE(op->mg.band_sweeps >= 0 && op->mg.band_sweeps <= 256, DM_ERR_INVALID_ARG, "band_sweeps out of range");
        DM_REQUIRE(op->mg.band_sweeps_coarse >= 0 && op->mg.band_sweeps_coarse <= 256, DM_ERR_INVALID_ARG,
                   "band_sweeps_coarse out of range");
        DM_REQUIRE(op->mg.band_brick >= 1, DM_ERR_INVALID_ARG, "band_brick must be >= 1");
        DM_REQUIRE(op->mg.krylov_ff == 0 || op->mg.krylov_ff == 1, DM_ERR_INVALID_ARG, "krylov_ff must be 0 or 1");
        DM_REQUIRE(op->mg.jacobi_sweeps >= 1 && op->mg.jacobi_sweeps <= 16, DM_ERR_INVALID_ARG,
                   "jacobi_sweeps must be in [1, 16]");
        DM_REQUIRE(op->mg.precision >= 0 && op->mg.precision <= 2, DM_ERR_INVALID_ARG, "unknown precision");
        DM_REQUIRE(op->mg.power_iters >= 1, DM_ERR_INVALID_ARG, "power_iters must be >= 1");
        DM_REQUIRE(op->mg.stencil_shape >= -1 && op->mg.stencil_shape < kStencilShapes, DM_ERR_INVALID_ARG,
                   "stencil_shape out of range");
        const char* ng = std::getenv("DMEIG_NO_GRAPHS");
        op->graphs = !(ng && ng[0] && ng[0] != '0');
        setup_operator(op.get());
    });
    if (st != DM_OK) return st;
    *out = op.release();
    return DM_OK;
}

void dm_operator_destroy(dm_operator* op) {
    if (!op) return;
    if (op->ctx) cudaStreamSynchronize(op->ctx->stream);
    delete op;
}

int dm_operator_num_levels(const dm_operator* op) { return op ? op->nlev : 0; }

int dm_operator_stencil_shape(const dm_operator* op, int level) {
    if (!op || level < 0 || level >= op->nlev) return -1;
    return op->ol[level].shape;
}

double dm_operator_get_omega(const dm_operator* op, int level, int scalar) {
    if (!op || level < 0 || level >= op->nlev) return 0.0;
    return scalar ? op->ol[level].omega_s : op->ol[level].omega;
}

dm_status dm_operator_set_omega(dm_operator* op, int level, int scalar, double omega) {
    if (!op || level < 0 || level >= op->nlev) return DM_ERR_INVALID_ARG;
    if (scalar) op->ol[level].omega_s = omega;
    else op->ol[level].omega = omega;
    // captured V-cycles hold the old weights
    if (op->vexec) { cudaGraphExecDestroy(op->vexec); op->vexec = nullptr; }
    if (op->sexec) { cudaGraphExecDestroy(op->sexec); op->sexec = nullptr; }
    return DM_OK;
}

dm_status dm_operator_apply(dm_operator* op, int level, const double* x, double* y, int on_device) {
    if (!op || !x || !y || level < 0 || level >= op->nlev) return DM_ERR_INVALID_ARG;
    return guarded(op->ctx, [&] {
        const Grid3& g = glv(op, level).g;
        DBuf<double> xp(3ll * g.np), yp(3ll * g.np);
        faces_in(op, level, x, on_device, xp.get());
        apply_vec64(op, level, xp.get(), yp.get());
        faces_out(op, level, yp.get(), y, on_device);
    });
}

dm_status dm_operator_apply_ff(dm_operator* op, const double* x, double* y, int on_device) {
    if (!op || !x || !y) return DM_ERR_INVALID_ARG;
    return guarded(op->ctx, [&] {
        const GeoLevel& g0 = glv(op, 0);
        DM_REQUIRE(op->mg.krylov_ff && g0.ff, DM_ERR_INVALID_ARG, "operator created with krylov_ff = 0");
        cudaStream_t s = op->ctx->stream;
        const long long n3 = 3ll * g0.g.np;
        DBuf<double> xp(n3), yp(n3);
        DBuf<float2> wf(std::max(g0.nflist, 1));
        faces_in(op, 0, x, on_device, xp.get());
        vec_apply_ff(g0.g, g0.tiles.get(), g0.ntiles, g0.ffA.get(), g0.ffL.get(), g0.ffV.get(), op->sigma, xp.get(),
                     g0.fmap.get(), wf.get(), s);
        zero(yp.get(), sizeof(double) * n3, s);
        ff_scatter<double>(g0.nflist, g0.flist.get(), 1.0, wf.get(), yp.get(), s);
        faces_out(op, 0, yp.get(), y, on_device);
    });
}

dm_status dm_operator_diagonal(dm_operator* op, int level, double* d, int on_device) {
    if (!op || !d || level < 0 || level >= op->nlev) return DM_ERR_INVALID_ARG;
    return guarded(op->ctx, [&] {
        const GeoLevel& g = glv(op, level);
        DBuf<double> dp(3ll * g.g.np);
        vec_diagonal(g.g, g.A.get(), g.L.get(), g.invV.get(), op->sigma, dp.get(), op->ctx->stream);
        faces_out(op, level, dp.get(), d, on_device);
    });
}

dm_status dm_operator_smooth(dm_operator* op, int level, const double* f, double* x, int on_device) {
    if (!op || !f || !x || level < 0 || level >= op->nlev) return DM_ERR_INVALID_ARG;
    return guarded(op->ctx, [&] {
        const GeoLevel& g = glv(op, level);
        const long long n3 = 3ll * g.g.np;
        DBuf<double> fp(n3), xp(n3), yp(n3);
        faces_in(op, level, f, on_device, fp.get());
        faces_in(op, level, x, on_device, xp.get());
        double* pads[3] = {fp.get(), xp.get(), yp.get()};
        cudaStream_t s = op->ctx->stream;
        const double om = op->ol[level].omega;
        double* u = op->band_u.get();
        auto run = [&](auto** p) {
            using T = std::remove_pointer_t<std::remove_reference_t<decltype(*p)>>;
            using TC = std::conditional_t<std::is_same<T, double>::value, double, float>;
            const VecOp<T, TC> o = vop<T, TC>(op, level);
            T* it = p[1];
            T* tmp = p[2];
            for (int k = 0; k < op->mg.jacobi_sweeps; ++k) {
                vec_stencil(o, ST_JACOBI, it, p[0], tmp, om, s);
                std::swap(it, tmp);
            }
            band_schwarz<T, TC>(Pick<T, TC>::bs(op->ol[level]), o.invD, g.g, g.band.get(), g.nband, p[0], it, u, om,
                                band_sweeps_of(op, level), level == 0, s);
            if (it != p[2]) DM_CUDA(cudaMemcpyAsync(p[2], it, sizeof(T) * (size_t)n3, cudaMemcpyDeviceToDevice, s));
        };
        if (op->mg.precision == DM_PREC_F64) run(reinterpret_cast<double**>(pads));
        else if (op->mg.precision == DM_PREC_F32)
            with_mg_vectors<float>(op, level, 3, pads, [&](float** p) { run(p); });
        else
            with_mg_vectors<__nv_bfloat16>(op, level, 3, pads, [&](__nv_bfloat16** p) { run(p); });
        faces_out(op, level, yp.get(), x, on_device);
    });
}

dm_status dm_operator_restrict(dm_operator* op, int level, const double* r, double* fc, int on_device) {
    if (!op || !r || !fc || level < 0 || level + 1 >= op->nlev) return DM_ERR_INVALID_ARG;
    return guarded(op->ctx, [&] {
        const GeoLevel& g = glv(op, level);
        const GeoLevel& gc = glv(op, level + 1);
        DBuf<double> rp(3ll * g.g.np), cp(3ll * gc.g.np);
        faces_in(op, level, r, on_device, rp.get());
        cudaStream_t s = op->ctx->stream;
        if (op->mg.precision == DM_PREC_F64) {
            face_restrict<double, double>(g.g, gc.g, gc.A.get(), rp.get(), cp.get(), gc.tiles.get(), gc.ntiles, s);
        } else {
            // the transfer weights are exact in any precision; run in the preconditioner's storage type
            const long long nf = 3ll * g.g.np, nc = 3ll * gc.g.np;
            const Domain df = g.vdom(), dc = gc.vdom();
            if (op->mg.precision == DM_PREC_F32) {
                DBuf<float> a(nf), b(nc);
                convert<float, double>(df, rp.get(), a.get(), s);
                face_restrict<float, float>(g.g, gc.g, gc.A32.get(), a.get(), b.get(), gc.tiles.get(), gc.ntiles, s);
                convert<double, float>(dc, b.get(), cp.get(), s);
                Sync::stream(s);
            } else {
                DBuf<__nv_bfloat16> a(nf), b(nc);
                convert<__nv_bfloat16, double>(df, rp.get(), a.get(), s);
                face_restrict<__nv_bfloat16, float>(g.g, gc.g, gc.A32.get(), a.get(), b.get(), gc.tiles.get(), gc.ntiles, s);
                convert<double, __nv_bfloat16>(dc, b.get(), cp.get(), s);
                Sync::stream(s);
            }
        }
        faces_out(op, level + 1, cp.get(), fc, on_device);
    });
}

dm_status dm_operator_prolong(dm_operator* op, int level, const double* ec, double* x, int on_device) {
    if (!op || !ec || !x || level < 0 || level + 1 >= op->nlev) return DM_ERR_INVALID_ARG;
    return guarded(op->ctx, [&] {
        const GeoLevel& g = glv(op, level);
        const GeoLevel& gc = glv(op, level + 1);
        DBuf<double> cp(3ll * gc.g.np), xp(3ll * g.g.np);
        faces_in(op, level + 1, ec, on_device, cp.get());
        faces_in(op, level, x, on_device, xp.get());
        cudaStream_t s = op->ctx->stream;
        if (op->mg.precision == DM_PREC_F64) {
            face_prolong_add<double, double>(g.g, gc.g, g.A.get(), cp.get(), xp.get(), g.tiles.get(), g.ntiles, s);
        } else {
            const long long nf = 3ll * g.g.np, nc = 3ll * gc.g.np;
            const Domain df = g.vdom(), dc = gc.vdom();
            if (op->mg.precision == DM_PREC_F32) {
                DBuf<float> a(nc), b(nf);
                convert<float, double>(dc, cp.get(), a.get(), s);
                convert<float, double>(df, xp.get(), b.get(), s);
                face_prolong_add<float, float>(g.g, gc.g, g.A32.get(), a.get(), b.get(), g.tiles.get(), g.ntiles, s);
                convert<double, float>(df, b.get(), xp.get(), s);
                Sync::stream(s);
            } else {
                DBuf<__nv_bfloat16> a(nc), b(nf);
                convert<__nv_bfloat16, double>(dc, cp.get(), a.get(), s);
                convert<__nv_bfloat16, double>(df, xp.get(), b.get(), s);
                face_prolong_add<__nv_bfloat16, float>(g.g, gc.g, g.A32.get(), a.get(), b.get(), g.tiles.get(), g.ntiles, s);
                convert<double, __nv_bfloat16>(df, b.get(), xp.get(), s);
                Sync::stream(s);
            }
        }
        faces_out(op, level, xp.get(), x, on_device);
    });
}

dm_status dm_operator_vcycle(dm_operator* op, const double* f, double* e, int on_device) {
    if (!op || !f || !e) return DM_ERR_INVALID_ARG;
    return guarded(op->ctx, [&] {
        const long long n3 = 3ll * glv(op, 0).g.np;
        DBuf<double> fp(n3), ep(n3);
        faces_in(op, 0, f, on_device, fp.get());
        precond_vec(op, fp.get(), ep.get());
        faces_out(op, 0, ep.get(), e, on_device);
    });
}

dm_status dm_operator_scalar_vcycle(dm_operator* op, const double* f, double* e, int on_device) {
    if (!op || !f || !e) return DM_ERR_INVALID_ARG;
    return guarded(op->ctx, [&] {
        const long long n1 = glv(op, 0).g.np;
        DBuf<double> fp(n1), ep(n1);
        cells_in(op, 0, f, on_device, fp.get());
        precond_scal(op, fp.get(), ep.get());
        cells_out(op, 0, ep.get(), e, on_device);
    });
}

dm_status dm_operator_solve(dm_operator* op, const double* b, double* x, int on_device, double tol, int restart,
                            int maxit, int* iters, double* relres) {
    if (!op || !b || !x || restart < 1 || restart > 120 || maxit < 1) return DM_ERR_INVALID_ARG;
    dm_status conv = DM_OK;
    const dm_status st = guarded(op->ctx, [&] {
        const long long n3 = 3ll * glv(op, 0).g.np;
        DBuf<double> bp(n3), xp(n3);
        faces_in(op, 0, b, on_device, bp.get());
        double rr = 0.0;
        const int it = solve_vec(op, bp.get(), xp.get(), tol, restart, maxit, &rr);
        if (iters) *iters = it;
        if (relres) *relres = rr;
        if (rr > 10.0 * tol) conv = DM_ERR_NO_CONVERGENCE;
        faces_out(op, 0, xp.get(), x, on_device);
    });
    return st != DM_OK ? st : conv;
}

dm_status dm_operator_project(dm_operator* op, const double* x, double* y, int on_device, double tol, int* iters) {
    if (!op || !x || !y) return DM_ERR_INVALID_ARG;
    return guarded(op->ctx, [&] {
        const long long n3 = 3ll * glv(op, 0).g.np;
        DBuf<double> xp(n3), yp(n3);
        faces_in(op, 0, x, on_device, xp.get());
        const int it = project(op, xp.get(), yp.get(), tol);
        if (iters) *iters = it;
        faces_out(op, 0, yp.get(), y, on_device);
    });
}

void dm_eig_params_default(dm_eig_params* p) {
    if (!p) return;
    p->sigma = 0.0;
    p->nev = 4;
    p->tol = 1e-10;
    p->inner_tol = 1e-9;
    p->proj_tol = 1e-12;
    p->basis = 0;
    p->max_restarts = 100;
    p->inner_restart = 40;
    p->inner_maxit = 400;
    p->seed = 1301;
    dm_mg_params_default(&p->mg);
    p->learned = nullptr;
    p->max_seconds = 0.0;
    p->rho_tol = 1e-8;
}

}  // extern "C"

namespace {

// k^2, rho, delta, rq of the eigenvectors in the padded FP64 columns X (ld = 3 np)
void certify_padded(dm_context* ctx, const GeoLevel& g0, int n, const double* X, double* k2_io, bool set_k2, double* rho,
                    double* delta, double* rq) {
    cudaStream_t s = ctx->stream;
    const long long n3 = 3ll * g0.g.np;
    const Domain D = g0.vdom(), Dc = g0.sdom();
    DBuf<double> kb(n3), ab(n3), dv(g0.g.np);
    const VecOp<double, double> o{g0.g, g0.A.get(), g0.L.get(), g0.invV.get(), nullptr, 0.0, 0};
    const double h = std::min(g0.g.hx, std::min(g0.g.hy, g0.g.hz));
    for (int i = 0; i < n; ++i) {
        const double* b = X + (size_t)i * n3;
        vec_stencil<double, double>(o, ST_APPLY, b, nullptr, kb.get(), 0.0, s);
        hadamard(D, g0.A.get(), b, ab.get(), s);
        // K b and A b vanish on closed faces, so the sums run over the open ones
        const double bkb = face_dot(ctx, g0, b, kb.get()), bab = face_dot(ctx, g0, b, ab.get());
        const double r = bkb / bab;
        if (rq) rq[i] = r;
        const double k2 = set_k2 ? r : k2_io[i];
        if (set_k2) k2_io[i] = r;
        const double abn = face_norm(ctx, g0, ab.get());
        axpby(D, -k2, ab.get(), 1.0, kb.get(), s);
        const double rn = face_norm(ctx, g0, kb.get());
        if (rho) rho[i] = rn / (std::fabs(k2) * abn);
        dm_div_a(g0.g, g0.A.get(), b, dv.get(), g0.tiles.get(), g0.ntiles, s);
        const double dn = norm2(ctx, Dc, dv.get());
        if (delta) delta[i] = dn * h / abn;
    }
}

__global__ void k_sign_fix(long long n, double* __restrict__ x, const double* __restrict__ sign) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        x[r] *= *sign;
}
// sign = +1 if the entry of largest magnitude is positive (first such entry on
// ties): per-block (value, index) maxima, then one block reduces them
constexpr int kSignBlocks = 304;
__device__ __forceinline__ void max_pair(double& bv, long long& bi, double v, long long i) {
    if (v > bv || (v == bv && i < bi)) {
        bv = v;
        bi = i;
    }
}
__device__ void block_max_pair(double& best, long long& idx) {
    __shared__ double bv[256];
    __shared__ long long bi[256];
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) max_pair(bv[threadIdx.x], bi[threadIdx.x], bv[threadIdx.x + s], bi[threadIdx.x + s]);
        __syncthreads();
    }
    best = bv[0];
    idx = bi[0];
}
__global__ void k_max_entry_partial(long long n, const double* __restrict__ x, double* __restrict__ pv,
                                    long long* __restrict__ pi) {
    double best = -1.0;
    long long idx = 0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        max_pair(best, idx, fabs(x[r]), r);
    block_max_pair(best, idx);
    if (threadIdx.x == 0) {
        pv[blockIdx.x] = best;
        pi[blockIdx.x] = idx;
    }
}
__global__ void k_max_entry_sign(int nb, const double* __restrict__ pv, const long long* __restrict__ pi,
                                 const double* __restrict__ x, double* __restrict__ sign) {
    double best = -1.0;
    long long idx = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) max_pair(best, idx, pv[b], pi[b]);
    block_max_pair(best, idx);
    if (threadIdx.x == 0) *sign = x[idx] < 0.0 ? -1.0 : 1.0;
}

}  // namespace

extern "C" {

dm_status dm_eigensolve(dm_context* ctx, const dm_geometry* geom, const dm_eig_params* prm, double* k2_out,
                        double* b_out, int b_on_device, dm_eig_report* report) {
    if (!ctx || !geom || !prm || !k2_out) return DM_ERR_INVALID_ARG;
    dm_status conv = DM_OK;
    bool stalled = false;     // kProjStallLimit projections reached the scalar solve's cap
    bool timed_out = false;   // the wall-clock limit p.max_seconds ran out
    const dm_status st = guarded(ctx, [&] {
        DM_CUDA(cudaSetDevice(ctx->device));
        cudaStream_t s = ctx->stream;
        const long long launches0 = ctx->launches;
        const dm_eig_params p = *prm;
        DM_REQUIRE(p.nev >= 1 && p.nev <= 40, DM_ERR_INVALID_ARG, "nev must be in [1, 40]");
        int m = p.basis > 0 ? p.basis : std::min(64, std::max(2 * p.nev + 10, 24));
        DM_REQUIRE(m >= p.nev + 2 && m <= 64, DM_ERR_INVALID_ARG, "basis must be in [nev + 2, 64]");
        DM_REQUIRE(p.max_seconds >= 0.0, DM_ERR_INVALID_ARG, "max_seconds must be >= 0");
        DM_REQUIRE(p.rho_tol >= 0.0, DM_ERR_INVALID_ARG, "rho_tol must be >= 0");
        DM_REQUIRE(p.tol > 0.0 && p.inner_tol > 0.0, DM_ERR_INVALID_ARG, "tol and inner_tol must be > 0");
        const double t_setup0 = now_s();
        auto out_of_time = [&] { return p.max_seconds > 0.0 && now_s() - t_setup0 > p.max_seconds; };
        dm_operator* op = nullptr;
        const dm_status cs = dm_operator_create(ctx, geom, p.sigma, &p.mg, &op);
        if (cs != DM_OK) throw Error(cs, std::string("operator setup: ") + ctx->err);
        std::unique_ptr<dm_operator, void (*)(dm_operator*)> opg(op, dm_operator_destroy);
        if (p.learned) {
            const dm_status ls = dm_operator_set_learned(op, p.learned);
            if (ls != DM_OK) throw Error(ls, std::string("learned: ") + ctx->err);
        }
        LaunchScope scope(ctx);
        const double t_solve0 = now_s();
        const GeoLevel& g0 = glv(op, 0);
        const Domain D = g0.vdom();
        const long long n = D.len();
        const double* a = g0.A.get();
        DBuf<double> Vb((size_t)(m + 1) * n), tmp((size_t)m * n), rhs(n), x(n);
        double* V = Vb.get();
        // With float-float Krylov work the basis also lives as float-float pairs
        // on the open faces (compact, even stride), and its Gram-Schmidt passes
        // run there on the FP32 pipes at HBM speed; the FP64 basis stays the
        // one the shifted solves, the Ritz vectors and the restarts use.
        const bool ffks = op->mg.krylov_ff && g0.ff;
        const long long nl = g0.nflist, nlp = (nl + 1) & ~1ll;
        DBuf<float2> Vff, tf, wf, wf2;
        if (ffks) {
            Vff.alloc((size_t)(m + 1) * nlp);
            tf.alloc(nlp);
            wf.alloc(nlp);
            wf2.alloc(nlp);
        }
        Grid3 gcf = g0.g;
        gcf.np = (int)nlp;
        const Domain Dc{gcf, nullptr, 0, 1};
        auto shadow = [&](int c0, int c1) {
            if (!ffks) return;
            for (int c = c0; c < c1; ++c)
                ff_gather(nl, g0.flist.get(), 1.0, V + (size_t)c * n, Vff.get() + (size_t)c * nlp, s);
        };
        std::vector<double> ffdots(2 * (size_t)m + 4), ffcoef(2 * (size_t)m + 4);
        // one Gram-Schmidt pass of w against V_0 .. V_j in the A inner product on
        // the float-float basis: h = V^T A w, w <- w - V h; returns (w^T A w
        // before, after) through wn2 (nullable) and the result
        auto ff_pass = [&](int j, double* w, std::vector<double>& h, double* wn2) -> double {
            const int nq = j + 1;
            hadamard(D, a, w, rhs.get(), s);
            ff_gather(nl, g0.flist.get(), 1.0, rhs.get(), tf.get(), s);
            ff_gather(nl, g0.flist.get(), 1.0, w, wf.get(), s);
            dcgs_dots(ctx->red, Dc, nq, Vff.get(), nlp, tf.get(), wf.get(), ffdots.data(), s);
            for (int c = 0; c < nq; ++c) h[c] = ffdots[c];
            if (wn2) *wn2 = ffdots[2 * nq + 1];
            for (int c = 0; c < nq; ++c) {
                ffcoef[c] = 0.0;
                ffcoef[nq + c] = h[c];
            }
            ffcoef[2 * nq] = 1.0;
            ffcoef[2 * nq + 1] = 0.0;
            dcgs_update(ctx->red, Dc, nq, Vff.get(), nlp, ffcoef.data(), tf.get(), wf.get(), wf2.get(), s);
            ff_scatter<double>(nl, g0.flist.get(), 1.0, wf2.get(), w, s);
            return face_dot(ctx, g0, w, w, a);
        };
        // start vector: seeded random on the open faces, projected, A-normalised
        fill_random(D, p.seed, a, rhs.get(), s);
        project(op, rhs.get(), V, p.proj_tol);
        {
            const double nv = face_norm(ctx, g0, V, a);
            DM_REQUIRE(nv > 0.0, DM_ERR_GEOMETRY, "start vector vanished under the projection (no open faces?)");
            scale_copy(D, 1.0 / nv, V, V, s);
        }
        shadow(0, 1);
        std::vector<double> H((size_t)(m + 1) * m, 0.0);
        auto Hat = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
        int k = 0, restarts = 0, outer = 0, inner_total = 0, proj_total = 0, nconv = 0, proj_capped = 0;
        std::vector<double> theta, Y, est;
        std::vector<int> order;
        // Ritz and inner tolerances in force: both tighten by 10 whenever the
        // Ritz estimates call the wanted pairs converged but their FP64
        // certificate rho (the residual of K b = k^2 A b itself) misses rho_tol
        double tol_eff = p.tol, inner_eff = p.inner_tol;
        int cert_retries = 0;
        // rho of the wanted Ritz pairs (|theta| order) from the current basis
        auto certify_wanted = [&](std::vector<double>& rho_out) {
            std::vector<double> Yw((size_t)m * p.nev), kk(p.nev);
            for (int c = 0; c < p.nev; ++c)
                for (int r = 0; r < m; ++r) Yw[(size_t)c * m + r] = Y[(size_t)r * m + order[c]];
            DBuf<double> Yd((size_t)m * p.nev);
            DM_CUDA(cudaMemcpyAsync(Yd.get(), Yw.data(), sizeof(double) * m * p.nev, cudaMemcpyHostToDevice, s));
            vgemm(D, m, p.nev, V, n, Yd.get(), m, tmp.get(), n, s);
            rho_out.assign(p.nev, 0.0);
            certify_padded(ctx, g0, p.nev, tmp.get(), kk.data(), true, rho_out.data(), nullptr, nullptr);
        };
        while (true) {
            for (int j = k; j < m; ++j) {
                if (out_of_time()) {
                    timed_out = true;
                    break;
                }
                double* vj = V + (size_t)j * n;
                hadamard(D, a, vj, rhs.get(), s);           // A v_j
                double rr = 0.0;
                inner_total += solve_vec(op, rhs.get(), x.get(), inner_eff, p.inner_restart, p.inner_maxit, &rr);
                double* w = V + (size_t)(j + 1) * n;
                const int pit = project(op, x.get(), w, p.proj_tol);   // w = P_DM (K - sigma A)^-1 A v_j
                proj_total += pit;
                ++outer;
                if (pit >= kProjMaxit && ++proj_capped >= kProjStallLimit) {
                    stalled = true;
                    break;
                }
                // A-orthogonalise against the basis: classical Gram-Schmidt,
                // repeated when the first pass cancelled most of w
                std::vector<double> h(j + 1);
                double wn2 = 0.0, bn2 = 0.0;
                if (ffks) {
                    bn2 = ff_pass(j, w, h, &wn2);
                } else {
                    mdot_self(ctx->red, D, j + 1, V, n, w, a, h.data(), &wn2, s);
                    bn2 = maxpy_norm(ctx->red, D, j + 1, V, n, w, a, s);
                }
                for (int i = 0; i <= j; ++i) Hat(i, j) += h[i];
                if (bn2 < 0.49 * wn2) {
                    if (ffks) {
                        bn2 = ff_pass(j, w, h, nullptr);
                    } else {
                        mdot(ctx->red, D, j + 1, V, n, w, a, h.data(), s);
                        bn2 = maxpy_norm(ctx->red, D, j + 1, V, n, w, a, s);
                    }
                    for (int i = 0; i <= j; ++i) Hat(i, j) += h[i];
                }
                const double beta = std::sqrt(std::max(bn2, 0.0));
                Hat(j + 1, j) = beta;
                DM_REQUIRE(beta > 0.0, DM_ERR_NO_CONVERGENCE, "Krylov space exhausted");
                scale_copy(D, 1.0 / beta, w, w, s);
                shadow(j + 1, j + 2);
            }
            // an interrupted expansion leaves no basis to extract pairs from
            if (stalled || timed_out) break;
            // Rayleigh-Ritz on the symmetrised projected matrix
            std::vector<double> Hs((size_t)m * m);
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < m; ++j) Hs[(size_t)i * m + j] = 0.5 * (Hat(i, j) + Hat(j, i));
            jacobi_eig(m, Hs, theta, Y);
            order.resize(m);
            std::iota(order.begin(), order.end(), 0);
            std::stable_sort(order.begin(), order.end(), [&](int x1, int x2) { return std::fabs(theta[x1]) > std::fabs(theta[x2]); });
            const double beta_m = Hat(m, m - 1);
            est.assign(m, 0.0);
            nconv = 0;
            for (int i = 0; i < m; ++i) est[i] = std::fabs(beta_m * Y[(size_t)(m - 1) * m + order[i]]);
            while (nconv < p.nev && est[nconv] <= tol_eff * std::fabs(theta[order[nconv]])) ++nconv;
            if (nconv >= p.nev && p.rho_tol > 0.0) {
                std::vector<double> rho_w;
                certify_wanted(rho_w);
                bool all_ok = true;
                for (double r : rho_w) all_ok = all_ok && r <= p.rho_tol;
                if (!all_ok && restarts < p.max_restarts && tol_eff > 1e-15) {
                    // The shifted solves were not accurate enough for the
                    // certificate, and the basis carries their error in its
                    // Arnoldi relation, which a thick restart would keep.  Tighten
                    // the tolerances (the Ritz one below the worst current
                    // estimate) and rebuild the basis from the sum of the wanted
                    // Ritz vectors with the tighter shifted solves.
                    double worst = 0.0;
                    for (int c = 0; c < p.nev; ++c)
                        worst = std::max(worst, est[c] / std::max(std::fabs(theta[order[c]]), 1e-300));
                    tol_eff = 0.1 * std::min(tol_eff, worst);
                    inner_eff = std::max(inner_eff * 0.1, 1e-13);
                    ++cert_retries;
                    std::vector<double> ones(p.nev, 1.0);
                    DBuf<double> od(p.nev);
                    DM_CUDA(cudaMemcpyAsync(od.get(), ones.data(), sizeof(double) * p.nev, cudaMemcpyHostToDevice, s));
                    vgemm(D, p.nev, 1, tmp.get(), n, od.get(), p.nev, V, n, s);   // tmp: the Ritz vectors
                    const double nv = face_norm(ctx, g0, V, a);
                    DM_REQUIRE(nv > 0.0, DM_ERR_NO_CONVERGENCE, "restart vector vanished");
                    scale_copy(D, 1.0 / nv, V, V, s);
                    shadow(0, 1);
                    std::fill(H.begin(), H.end(), 0.0);
                    k = 0;
                    ++restarts;
                    Sync::stream(s);
                    continue;
                }
            }
            if (nconv >= p.nev || restarts >= p.max_restarts) break;
            // thick restart: keep the pk wanted Ritz vectors
            const int pk = std::min(m - 1, p.nev + (m - p.nev) / 2);
            std::vector<double> Yk((size_t)m * pk);
            for (int c = 0; c < pk; ++c)
                for (int r = 0; r < m; ++r) Yk[(size_t)c * m + r] = Y[(size_t)r * m + order[c]];
            DBuf<double> Yd((size_t)m * pk);
            DM_CUDA(cudaMemcpyAsync(Yd.get(), Yk.data(), sizeof(double) * m * pk, cudaMemcpyHostToDevice, s));
            vgemm(D, m, pk, V, n, Yd.get(), m, tmp.get(), n, s);
            DM_CUDA(cudaMemcpyAsync(V, tmp.get(), sizeof(double) * pk * n, cudaMemcpyDeviceToDevice, s));
            DM_CUDA(cudaMemcpyAsync(V + (size_t)pk * n, V + (size_t)m * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            shadow(0, pk + 1);
            std::fill(H.begin(), H.end(), 0.0);
            for (int c = 0; c < pk; ++c) {
                Hat(c, c) = theta[order[c]];
                Hat(pk, c) = beta_m * Y[(size_t)(m - 1) * m + order[c]];
            }
            k = pk;
            ++restarts;
            Sync::stream(s);
        }
        const int nev = p.nev;
        if (stalled || timed_out) {
            // no pair is returned: k^2 are NaN, b_out is left untouched
            for (int c = 0; c < nev; ++c) k2_out[c] = std::numeric_limits<double>::quiet_NaN();
            conv = timed_out ? DM_ERR_TIMEOUT : DM_ERR_NO_CONVERGENCE;
            if (report) {
                *report = dm_eig_report{};
                report->outer_iters = outer;
                report->restarts = restarts;
                report->inner_iters = inner_total;
                report->proj_iters = proj_total;
                report->mg_levels = op->nlev;
                report->mg_complexity = op->complexity;
                report->rho_max = std::numeric_limits<double>::quiet_NaN();
                report->delta_max = std::numeric_limits<double>::quiet_NaN();
                report->setup_seconds = t_solve0 - t_setup0;
                report->solve_seconds = now_s() - t_solve0;
                report->kernel_launches = ctx->launches - launches0;
                report->learned_applied = op->learned_applied;
                report->learned_fallbacks = op->learned_fallbacks;
            }
            Sync::stream(s);
            return;
        }
        // Ritz vectors of the wanted pairs, in the order of |theta|
        std::vector<double> Yw((size_t)m * nev);
        for (int c = 0; c < nev; ++c)
            for (int r = 0; r < m; ++r) Yw[(size_t)c * m + r] = Y[(size_t)r * m + order[c]];
        DBuf<double> Yd((size_t)m * nev), sign(1), pv(kSignBlocks);
        DBuf<long long> pi(kSignBlocks);
        DM_CUDA(cudaMemcpyAsync(Yd.get(), Yw.data(), sizeof(double) * m * nev, cudaMemcpyHostToDevice, s));
        vgemm(D, m, nev, V, n, Yd.get(), m, tmp.get(), n, s);
        std::vector<double> k2(nev), rho(nev), delta(nev), rq(nev);
        for (int c = 0; c < nev; ++c) {
            double* b = tmp.get() + (size_t)c * n;
            const double nb = face_norm(ctx, g0, b, a);
            scale_copy(D, 1.0 / nb, b, b, s);
            launch("k_max_entry_partial", k_max_entry_partial, kSignBlocks, 256, 0, s, n, (const double*)b, pv.get(),
                   pi.get());
            launch("k_max_entry_sign", k_max_entry_sign, 1, 256, 0, s, kSignBlocks, (const double*)pv.get(),
                   (const long long*)pi.get(), (const double*)b, sign.get());
            launch("k_sign_fix", k_sign_fix, (int)std::min<long long>((n + 255) / 256, 1216), 256, 0, s, n, b, sign.get());
        }
        certify_padded(ctx, g0, nev, tmp.get(), k2.data(), true, rho.data(), delta.data(), rq.data());
        if (p.rho_tol > 0.0) {
            // the converged prefix (|theta| order) also needs its certificate
            int nc = 0;
            while (nc < nconv && rho[nc] <= p.rho_tol) ++nc;
            nconv = nc;
        }
        // ascending k^2
        std::vector<int> asc(nev);
        std::iota(asc.begin(), asc.end(), 0);
        std::stable_sort(asc.begin(), asc.end(), [&](int x1, int x2) { return k2[x1] < k2[x2]; });
        double rho_max = 0.0, delta_max = 0.0;
        for (int c = 0; c < nev; ++c) {
            k2_out[c] = k2[asc[c]];
            rho_max = std::max(rho_max, rho[asc[c]]);
            delta_max = std::max(delta_max, delta[asc[c]]);
        }
        if (b_out) {
            // host output: one staging buffer, each vector unpacked into it and
            // copied out in stream order (a pinned destination copies at link speed)
            const size_t nf = (size_t)natural_faces(g0.g);
            DBuf<double> t;
            if (!b_on_device) t.alloc(nf, false);
            for (int c = 0; c < nev; ++c) {
                const double* src = tmp.get() + (size_t)asc[c] * n;
                if (b_on_device) {
                    unpack_faces(g0.g, src, b_out + c * nf, s);
                } else {
                    unpack_faces(g0.g, src, t.get(), s);
                    DM_CUDA(cudaMemcpyAsync(b_out + c * nf, t.get(), sizeof(double) * nf, cudaMemcpyDeviceToHost, s));
                }
            }
            Sync::stream(s);
        }
        Sync::stream(s);
        if (nconv < nev) conv = DM_ERR_NO_CONVERGENCE;
        if (report) {
            report->n_converged = nconv;
            report->outer_iters = outer;
            report->restarts = restarts;
            report->inner_iters = inner_total;
            report->proj_iters = proj_total;
            report->mg_levels = op->nlev;
            report->mg_complexity = op->complexity;
            report->rho_max = rho_max;
            report->delta_max = delta_max;
            report->setup_seconds = t_solve0 - t_setup0;
            report->solve_seconds = now_s() - t_solve0;
            report->kernel_launches = ctx->launches - launches0;
            report->learned_applied = op->learned_applied;
            report->learned_fallbacks = op->learned_fallbacks;
        }
    });
    if (st == DM_OK && stalled)
        ctx->err = "projection: the scalar solve of P_DM reached its iteration cap (" + std::to_string(kProjMaxit) +
                   ") in " + std::to_string(kProjStallLimit) + " projections; no eigenpair is returned";
    if (st == DM_OK && timed_out)
        ctx->err = "eigensolve: the wall-clock limit of " + std::to_string(prm->max_seconds) +
                   " s ran out; no eigenpair is returned";
    return st != DM_OK ? st : conv;
}

// ---------------------------------------------------------------------------
// operator apply without any allocation
// ---------------------------------------------------------------------------

}  // extern "C"

namespace {

// Scratch of dm_operator_apply_noalloc: the padded input and output vectors of
// one call.  It lives in the library's own device image, so every GPU that
// loads the library holds it until the process exits.
constexpr long long kNoAllocDoubles = 6ll * 1024 * 1024;   // 48 MiB
__device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Device address of g_noalloc_scratch on `dev` (the current device), looked
// up once per device: in host code the symbol names a host-side stand-in, not
// device memory, so it must never be passed to a kernel directly.
double* noalloc_scratch(int dev) {
    static std::mutex mu;
    static double* addr[128] = {};
    DM_REQUIRE(dev >= 0 && dev < 128, DM_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            throw Error(DM_ERR_CUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
        addr[dev] = static_cast<double*>(p);
    }
    return addr[dev];
}

}  // namespace

extern "C" {

dm_status dm_operator_apply_noalloc(dm_operator* op, int level, const double* x, double* y) {
    if (!op || !x || !y || level < 0 || level >= op->nlev) return DM_ERR_INVALID_ARG;
    return guarded(op->ctx, [&] {
        // event timing would create CUDA events, and this call creates nothing:
        // its launches are never traced (the context's tracer is left as it is)
        UntracedScope untraced;
        DM_CUDA(cudaSetDevice(op->ctx->device));
        const GeoLevel& g = glv(op, level);
        const long long n3 = 3ll * g.g.np;
        if (2 * n3 > kNoAllocDoubles)
            throw Error(DM_ERR_INVALID_ARG, "dm_operator_apply_noalloc: level " + std::to_string(level) + " needs " +
                                                std::to_string(2 * n3) + " doubles of scratch; the static scratch holds " +
                                                std::to_string(kNoAllocDoubles) + " (use dm_operator_apply)");
        cudaStream_t s = op->ctx->stream;
        double* xp = noalloc_scratch(op->ctx->device);
        double* yp = xp + n3;
        // the scratch keeps the previous call's contents: the padded input must
        // start at zero (ghost and non-face entries are read by the stencil)
        DM_CUDA(cudaMemsetAsync(xp, 0, sizeof(double) * (size_t)n3, s));
        pack_faces(g.g, x, xp, s);
        launch("k_mask_open", k_mask_open, (int)std::min<long long>((n3 + 255) / 256, 1216), 256, 0, s, n3, g.A.get(),
               xp);
        vec_apply_dense_f64(g.g, g.A.get(), g.L.get(), g.invV.get(), op->sigma, xp, yp, s);
        unpack_faces(g.g, yp, y, s);
        DM_CUDA(cudaStreamSynchronize(s));
    });
}

// ---------------------------------------------------------------------------
// learned smoother
// ---------------------------------------------------------------------------

dm_status dm_learned_create(dm_context* ctx, unsigned long long seed, dm_learned** out) {
    if (!ctx || !out) return DM_ERR_INVALID_ARG;
    *out = nullptr;
    auto net = std::make_unique<dm_learned>();
    const dm_status st = guarded(ctx, [&] {
        net->ctx = ctx;
        net->net.init_params();
        // He-normal initialisation (fan-in 27 * Cin); the last layer scaled by 0.1
        std::mt19937_64 rng(seed);
        std::normal_distribution<double> nd(0.0, 1.0);
        std::vector<float> w(LearnedNet::n_params());
        auto fill = [&](size_t off, size_t n, int cin, double extra) {
            const double sd = std::sqrt(2.0 / (27.0 * cin)) * extra;
            for (size_t t = 0; t < n; ++t) w[off + t] = (float)(nd(rng) * sd);
        };
        fill(0, LearnedNet::n1(), LearnedNet::CIN_, 1.0);
        fill(LearnedNet::off2(), LearnedNet::n2(), LearnedNet::HID, 1.0);
        fill(LearnedNet::off3(), LearnedNet::n3(), LearnedNet::HID, 0.1);
        DM_CUDA(cudaMemcpyAsync(net->net.W.get(), w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, ctx->stream));
        Sync::stream(ctx->stream);
    });
    if (st != DM_OK) return st;
    *out = net.release();
    return DM_OK;
}

void dm_learned_destroy(dm_learned* net) {
    if (!net) return;
    if (net->ctx) cudaStreamSynchronize(net->ctx->stream);
    delete net;
}

long long dm_learned_num_params(void) { return (long long)LearnedNet::n_params(); }

dm_status dm_learned_get_weights(const dm_learned* net, float* w) {
    if (!net || !w) return DM_ERR_INVALID_ARG;
    return guarded(net->ctx, [&] {
        DM_CUDA(cudaMemcpyAsync(w, net->net.W.get(), sizeof(float) * LearnedNet::n_params(), cudaMemcpyDeviceToHost,
                                net->ctx->stream));
        Sync::stream(net->ctx->stream);
    });
}

dm_status dm_learned_set_weights(dm_learned* net, const float* w) {
    if (!net || !w) return DM_ERR_INVALID_ARG;
    return guarded(net->ctx, [&] {
        DM_CUDA(cudaMemcpyAsync(net->net.W.get(), w, sizeof(float) * LearnedNet::n_params(), cudaMemcpyHostToDevice,
                                net->ctx->stream));
        Sync::stream(net->ctx->stream);
        net->net.step = 0;
        zero(net->net.M1.get(), sizeof(float) * LearnedNet::n_params(), net->ctx->stream);
        zero(net->net.M2.get(), sizeof(float) * LearnedNet::n_params(), net->ctx->stream);
    });
}

dm_status dm_learned_apply(dm_learned* net, const dm_geometry* geom, const double* r, double* y, int on_device) {
    if (!net || !geom || !r || !y) return DM_ERR_INVALID_ARG;
    return guarded(net->ctx, [&] {
        dm_context* ctx = net->ctx;
        cudaStream_t s = ctx->stream;
        const GeoLevel& g0 = *geom->lv[0];
        const long long n3 = 3ll * g0.g.np;
        const size_t nf = (size_t)natural_faces(g0.g);
        DBuf<double> rp(n3), yp(n3), tmp;
        const double* d = nullptr;
        stage_in(ctx, r, on_device, nf, tmp, &d);
        pack_faces(g0.g, d, rp.get(), s);
        launch("k_mask_open", k_mask_open, (int)std::min<long long>((n3 + 255) / 256, 1216), 256, 0, s, n3, g0.A.get(),
               rp.get());
        DBuf<int> cnt(1);
        const long long nopen = count_positive(n3, g0.A.get(), cnt.get(), s);
        const double ss = sumsq<double>(n3, rp.get(), s);
        if (ss > 0.0 && nopen > 0) {
            const double scale = std::sqrt(ss / (double)nopen);
            const double h = std::min(g0.g.hx, std::min(g0.g.hy, g0.g.hz));
            net->net.alloc(g0.g);
            net->net.features(g0.A.get(), g0.V.get(), 1.0 / scale, rp.get(), 0, s);
            net->net.forward(s);
            net->net.check(s);
            net->net.add_correction<double>(g0.A.get(), scale * h * h, yp.get(), s);
        }
        if (on_device) {
            unpack_faces(g0.g, yp.get(), y, s);
            Sync::stream(s);
        } else {
            DBuf<double> t(nf, false);
            unpack_faces(g0.g, yp.get(), t.get(), s);
            stage_out(ctx, t.get(), y, 0, nf);
        }
    });
}

dm_status dm_learned_loss_grad(dm_learned* net, const dm_geometry* geom, const float* X, const float* E, float* loss,
                               float* grad) {
    if (!net || !geom || !X || !E) return DM_ERR_INVALID_ARG;
    return guarded(net->ctx, [&] {
        dm_context* ctx = net->ctx;
        cudaStream_t s = ctx->stream;
        const GeoLevel& g0 = *geom->lv[0];
        const size_t nn = (size_t)(g0.g.nx + 1) * (g0.g.ny + 1) * (g0.g.nz + 1);
        DBuf<float> xd(nn * LearnedNet::CIN_, false), ed(nn * LearnedNet::COUT_, false);
        DM_CUDA(cudaMemcpyAsync(xd.get(), X, sizeof(float) * nn * LearnedNet::CIN_, cudaMemcpyHostToDevice, s));
        DM_CUDA(cudaMemcpyAsync(ed.get(), E, sizeof(float) * nn * LearnedNet::COUT_, cudaMemcpyHostToDevice, s));
        LearnedNet& L = net->net;
        L.alloc(g0.g);
        L.set_X(xd.get(), s);
        L.set_E(ed.get(), s);
        L.forward(s);
        DBuf<int> cnt(1);
        const long long nopen = count_positive(3ll * g0.g.np, g0.A.get(), cnt.get(), s);
        const float l = L.loss(g0.A.get(), (double)nopen, s);
        L.backward(s);
        L.check(s);
        if (loss) *loss = l;
        if (grad) {
            DM_CUDA(cudaMemcpyAsync(grad, L.G.get(), sizeof(float) * LearnedNet::n_params(), cudaMemcpyDeviceToHost, s));
        }
        Sync::stream(s);
    });
}

dm_status dm_learned_train(dm_learned* net, dm_operator* op, int runs, int epochs, float lr, unsigned long long seed,
                           float* loss_history) {
    if (!net || !op || runs < 1 || epochs < 1 || !(lr > 0.f)) return DM_ERR_INVALID_ARG;
    return guarded(op->ctx, [&] {
        dm_context* ctx = op->ctx;
        cudaStream_t s = ctx->stream;
        GeoLevel& g0 = *const_cast<dm_geometry*>(op->geom)->lv[0];
        const Domain D = g0.vdom();
        const long long n3 = D.len();
        const double h = std::min(g0.g.hx, std::min(g0.g.hy, g0.g.hz));
        // 1. residuals the plain V-cycle leaves: for Krylov directions v of
        //    FGMRES-like sequences, z = V-cycle(v), r = v - (K - sigma A) z
        const int dirs = 8;
        std::vector<DBuf<float>> R;
        std::vector<double> scales;
        DBuf<double> v((size_t)(dirs + 1) * n3), z(n3), r(n3);
        std::unique_ptr<LearnedNet> keep = std::move(op->lnet);   // plain V-cycle while sampling
        for (int run = 0; run < runs; ++run) {
            fill_random(D, seed + 7919ull * run, g0.A.get(), v.get(), s);
            double nv = norm2(ctx, D, v.get());
            scale_copy(D, 1.0 / nv, v.get(), v.get(), s);
            for (int j = 0; j < dirs; ++j) {
                double* vj = v.get() + (size_t)j * n3;
                precond_vec(op, vj, z.get());
                apply_vec64(op, 0, z.get(), r.get());          // r = (K - sigma A) z
                axpby(D, 1.0, vj, -1.0, r.get(), s);          // r = v - (K - sigma A) z
                const double rs = std::sqrt(sumsq<double>(n3, r.get(), s) / (double)std::max(op->nopen0, 1ll));
                if (rs > 0.0) {
                    R.emplace_back(n3);
                    convert<float, double>(D, r.get(), R.back().get(), s);
                    scales.push_back(rs);
                }
                // next direction: (K - sigma A) z orthonormalised against the previous ones
                double* w = v.get() + (size_t)(j + 1) * n3;
                apply_vec64(op, 0, z.get(), w);
                std::vector<double> hh(j + 1);
                mdot(ctx->red, D, j + 1, v.get(), n3, w, nullptr, hh.data(), s);
                maxpy(ctx->red, D, j + 1, v.get(), n3, hh.data(), w, s);
                const double nw = norm2(ctx, D, w);
                if (!(nw > 0.0)) break;
                scale_copy(D, 1.0 / nw, w, w, s);
            }
        }
        op->lnet = std::move(keep);
        DM_REQUIRE(!R.empty(), DM_ERR_NO_CONVERGENCE, "learned training: no samples");
        // 2. Adam on the residual objective 0.5 |r / RMS(r) - K h^2 N(r)|^2 / #open
        //    (FP32 operator), samples in a seeded order every epoch
        {
            std::lock_guard<std::mutex> lock(const_cast<dm_geometry*>(op->geom)->mu);
            ensure_f32(g0, s);
        }
        const VecOp<float, float> o32{g0.g, g0.A32.get(), g0.L32.get(), g0.invV32.get(), nullptr, op->sigma, 0,
                                      g0.tiles.get(), g0.ntiles, nullptr, 0, 0};
        DBuf<float> ybuf(n3), kbuf(n3);
        LearnedNet& L = net->net;
        L.alloc(g0.g);
        std::mt19937_64 rng(seed ^ 0x5bd1e995ull);
        std::vector<int> order(R.size());
        std::iota(order.begin(), order.end(), 0);
        for (int ep = 0; ep < epochs; ++ep) {
            std::shuffle(order.begin(), order.end(), rng);
            double tot = 0.0;
            for (int k : order) {
                L.features(g0.A.get(), g0.V.get(), 1.0 / scales[k], R[k].get(), 1, s);
                L.forward(s);
                tot += L.residual_loss(o32, g0.A.get(), R[k].get(), 1.0 / scales[k], h * h, ybuf.get(), kbuf.get(),
                                       (double)op->nopen0, s);
                L.backward(s);
                L.adam(lr, s);
            }
            if (loss_history) loss_history[ep] = (float)(tot / (double)order.size());
            L.check(s);
        }
        Sync::stream(s);
    });
}

dm_status dm_learned_train_step(dm_learned* net, dm_operator* op, const double* r, int on_device, float lr,
                                float* loss, float* grad) {
    if (!net || !op || !r || !(lr >= 0.f)) return DM_ERR_INVALID_ARG;
    return guarded(op->ctx, [&] {
        dm_context* ctx = op->ctx;
        cudaStream_t s = ctx->stream;
        GeoLevel& g0 = *const_cast<dm_geometry*>(op->geom)->lv[0];
        const long long n3 = 3ll * g0.g.np;
        const double h = std::min(g0.g.hx, std::min(g0.g.hy, g0.g.hz));
        DBuf<double> rp(n3);
        faces_in(op, 0, r, on_device, rp.get());
        const double ss = sumsq<double>(n3, rp.get(), s);
        DM_REQUIRE(ss > 0.0 && op->nopen0 > 0, DM_ERR_INVALID_ARG, "learned train step: zero residual");
        const double rms = std::sqrt(ss / (double)op->nopen0);
        {
            std::lock_guard<std::mutex> lock(const_cast<dm_geometry*>(op->geom)->mu);
            ensure_f32(g0, s);
        }
        DBuf<float> r32(n3), ybuf(n3), kbuf(n3);
        convert<float, double>(g0.vdom(), rp.get(), r32.get(), s);
        const VecOp<float, float> o32{g0.g, g0.A32.get(), g0.L32.get(), g0.invV32.get(), nullptr, op->sigma, 0,
                                      g0.tiles.get(), g0.ntiles, nullptr, 0, 0};
        LearnedNet& L = net->net;
        L.alloc(g0.g);
        L.features(g0.A.get(), g0.V.get(), 1.0 / rms, r32.get(), 1, s);
        L.forward(s);
        const float l = L.residual_loss(o32, g0.A.get(), r32.get(), 1.0 / rms, h * h, ybuf.get(), kbuf.get(),
                                        (double)op->nopen0, s);
        L.backward(s);
        L.check(s);
        if (loss) *loss = l;
        if (grad) {
            DM_CUDA(cudaMemcpyAsync(grad, L.G.get(), sizeof(float) * LearnedNet::n_params(), cudaMemcpyDeviceToHost, s));
            Sync::stream(s);
        }
        L.adam(lr, s);
        Sync::stream(s);
    });
}

dm_status dm_operator_set_learned(dm_operator* op, const dm_learned* net) {
    if (!op) return DM_ERR_INVALID_ARG;
    return guarded(op->ctx, [&] {
        op->learned_streak = 0;
        if (!net) {
            op->lnet.reset();
            return;
        }
        auto ln = std::make_unique<LearnedNet>();
        ln->init_params();
        DM_CUDA(cudaMemcpyAsync(ln->W.get(), net->net.W.get(), sizeof(float) * LearnedNet::n_params(),
                                cudaMemcpyDeviceToDevice, op->ctx->stream));
        ln->alloc(glv(op, 0).g);
        Sync::stream(op->ctx->stream);
        op->lnet = std::move(ln);
    });
}

dm_status dm_eigensolve_batched(dm_context* ctx, int n, dm_batch_item* items, int streams) {
    if (!ctx || n < 0 || (n > 0 && !items) || streams < 1) return DM_ERR_INVALID_ARG;
    if (n == 0) return DM_OK;
    // largest work first: faces x modes
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    auto work = [&](int i) -> double {
        const dm_geometry* g = items[i].geom;
        if (!g || g->lv.empty()) return 0.0;
        return (double)natural_faces(g->lv[0]->g) * std::max(1, items[i].params.nev);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
    // Stencil tile shapes are tuned here, before the workers start: one
    // operator per distinct fine grid and precision on the calling context, so
    // that the autotuner times its candidates with the GPU otherwise idle; the
    // workers then find every shape in the cache.
    {
        std::vector<std::array<int, 4>> seen;
        for (int i = 0; i < n; ++i) {
            const dm_batch_item& it = items[order[i]];
            if (!it.geom || it.geom->lv.empty() || !it.params.mg.autotune || it.params.mg.stencil_shape >= 0)
                continue;
            const Grid3& g0 = it.geom->lv[0]->g;
            const std::array<int, 4> key{g0.nx, g0.ny, g0.nz, it.params.mg.precision};
            if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
            seen.push_back(key);
            bool cached = false;
            for (const auto& kv : ctx->tuned) cached |= kv.first == key;
            if (cached) continue;
            dm_operator* op = nullptr;
            if (dm_operator_create(ctx, it.geom, it.params.sigma, &it.params.mg, &op) == DM_OK) dm_operator_destroy(op);
        }
        ctx->err.clear();
    }
    const int nw = std::min(streams, n);
    std::vector<dm_context*> sub(nw, nullptr);
    for (int w = 0; w < nw; ++w) {
        const dm_status st = dm_context_create(ctx->device, nullptr, &sub[w]);
        if (st != DM_OK) {
            for (int u = 0; u < w; ++u) dm_context_destroy(sub[u]);
            ctx->err = "batched: cannot create worker stream";
            return st;
        }
        sub[w]->tuned = ctx->tuned;
    }
    std::atomic<int> next{0};
    auto worker = [&](int w) {
        cudaSetDevice(ctx->device);
        while (true) {
            const int k = next.fetch_add(1);
            if (k >= n) break;
            dm_batch_item& it = items[order[k]];
            if (!it.geom || !it.k2_out) {
                it.status = DM_ERR_INVALID_ARG;
                continue;
            }
            it.status = dm_eigensolve(sub[w], it.geom, &it.params, it.k2_out, it.b_out, it.b_on_device, &it.report);
        }
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < nw; ++w) pool.emplace_back(worker, w);
    worker(0);
    for (auto& t : pool) t.join();
    dm_status first = DM_OK;
    std::string msg;
    for (int w = 0; w < nw; ++w) {
        ctx->launches += sub[w]->launches;
        if (msg.empty() && !sub[w]->err.empty()) msg = sub[w]->err;
        for (const auto& kv : sub[w]->tuned) {
            bool have = false;
            for (const auto& c : ctx->tuned) have |= c.first == kv.first;
            if (!have) ctx->tuned.push_back(kv);
        }
        dm_context_destroy(sub[w]);
    }
    for (int i = 0; i < n; ++i)
        if (items[i].status != DM_OK && first == DM_OK) first = (dm_status)items[i].status;
    ctx->err = msg;
    return first;
}

dm_status dm_certify(dm_context* ctx, const dm_geometry* geom, int n, const double* k2, const double* b, int on_device,
                     double* rho, double* delta, double* rq) {
    if (!ctx || !geom || !b || !k2 || n < 1) return DM_ERR_INVALID_ARG;
    return guarded(ctx, [&] {
        const GeoLevel& g0 = *geom->lv[0];
        cudaStream_t s = ctx->stream;
        const long long n3 = 3ll * g0.g.np;
        const size_t nf = (size_t)natural_faces(g0.g);
        DBuf<double> X((size_t)n * n3);
        for (int i = 0; i < n; ++i) {
            DBuf<double> tmpb;
            const double* d = nullptr;
            stage_in(ctx, b + i * nf, on_device, nf, tmpb, &d);
            pack_faces(g0.g, d, X.get() + (size_t)i * n3, s);
            Sync::stream(s);
        }
        std::vector<double> kk(k2, k2 + n);
        certify_padded(ctx, g0, n, X.get(), kk.data(), false, rho, delta, rq);
    });
}

}  // extern "C"
