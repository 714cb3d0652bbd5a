// xy_api.cu -- C-ABI of the Cartesian transverse grid (3D+1; declared in
// include/fcn.h, "Cartesian transverse grid").  Host-side orchestration
// only: argument checks, device buffers, the pivot tables of the two axes,
// variant timing and CUDA-graph capture of the z-loop.  Every arithmetic
// step runs in the row kernels (row_kernel.cuh: nonlinear half steps and the
// FFT along tau of every (x, y) row), the line kernels (xy_kernel.cu: the x
// and the y Crank-Nicolson factors) and reduce.cu (diagnostics).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/fcn.h"
#include "fcn_device.cuh"
#include "fcn_host.h"

using namespace fcn;

struct fcn_xy_ctx {
    int prec = FCN_FP64;
    cudaStream_t st = nullptr;      // launch stream
    cudaStream_t cap = nullptr;     // capture stream (graphs replay on st)
    fcn_grid_xy g{};
    fcn_params p{};
    fcn_grid rg{};                  // the time grid in radial form (nr, r_max unused)
    void *field = nullptr;          // [nx][ny][nt] complex, time domain between calls
    void *rho = nullptr;            // [nx][ny][nt] real, rho of the last half step
    void *stage = nullptr;          // FP64 staging for host transfers
    double *stats = nullptr;        // [nx*ny][NSTAT]
    double *red = nullptr;          // [16]
    double *host_red = nullptr;     // pinned [16]
    const void *tw = nullptr;
    const void *tw1 = nullptr;   // twiddles of FFT plan 1 (FP32, Nt >= 256), or null
    // pivot tables of the current dz: x lines (no dispersion), y lines
    uint64_t tab_dz = 0;
    void *tab_x = nullptr, *tab_y = nullptr;
    std::map<uint64_t, cudaGraphExec_t> graphs;   // 8 (x, y, mid) steps per dz
    double z = 0.0;
    int64_t steps = 0;
    bool has_field = false;
    int row_var = 0, line_var = 0;
    bool tuned = false;
    int force_row = -1, force_line = -1;
    bool profiling = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_events;
    double prof_ms[FCN_XY_PROF_KINDS] = {0};
    int64_t prof_n[FCN_XY_PROF_KINDS] = {0};
    std::string err = "no error";
    int64_t rows() const { return (int64_t)g.nx * g.ny; }
    int64_t points() const { return rows() * g.nt; }
};

namespace {

std::string g_xy_create_error = "no error";
std::mutex g_xy_mu;

constexpr int OPS_HEAD = OP_NL | OP_FFT;
constexpr int OPS_MID = OP_IFFT | OP_NL | OP_NL2 | OP_FFT;
constexpr int OPS_TAIL = OP_IFFT | OP_NL | OP_RHO | OP_STATS;

int fail(fcn_xy_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    else g_xy_create_error = msg;
    return code;
}

int cuda_fail(fcn_xy_ctx *c, cudaError_t e, const char *what) {
    return fail(c, FCN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

uint64_t bits(double v) {
    uint64_t k;
    std::memcpy(&k, &v, sizeof k);
    return k;
}

size_t csize(int prec) { return prec == FCN_FP64 ? 16 : 8; }
size_t rsize(int prec) { return prec == FCN_FP64 ? 8 : 4; }

// s of an axis with spacing h and the dispersion coefficients (delta_q =
// dk q^2 on the y lines' diagonal, or the exact factor exp(2 i disp q^2)).
void line_coefs(const fcn_xy_ctx *ctx, double dz, double h, double *s, double *dk, double *disp) {
    double k0, dtau, domega;
    hostx::consts(ctx->rg, ctx->p, &k0, &dtau, &domega);
    *s = (ctx->p.flags & FCN_DIFFRACTION) ? dz / (4.0 * k0 * h * h) : 0.0;
    const double d = (ctx->p.flags & FCN_DISPERSION) ? ctx->p.k2 * dz / 4.0 * domega * domega : 0.0;
    const bool exact = (ctx->p.flags & FCN_EXACT_DISPERSION) != 0;
    *dk = exact ? 0.0 : d;
    *disp = exact ? d : 0.0;
}

double dx_of(const fcn_xy_ctx *ctx) { return ctx->g.x_width / double(ctx->g.nx - 1); }
double dy_of(const fcn_xy_ctx *ctx) { return ctx->g.y_width / double(ctx->g.ny - 1); }

template <typename T>
RowArgs<T> row_args(fcn_xy_ctx *ctx, void *field, int ops, double dz) {
    RowArgs<T> a;
    a.field = (cx<T> *)field;
    a.tw = (const cx<T> *)ctx->tw;
    a.tw1 = (const cx<T> *)ctx->tw1;
    a.rho = (T *)ctx->rho;
    a.stats = ctx->stats;
    a.nr = (int)ctx->rows();
    a.nt = ctx->g.nt;
    a.ops = ops;
    a.variant = ctx->row_var;
    a.nl = hostx::nl<T>(ctx->rg, ctx->p, 0.5 * dz);
    return a;
}

// axis 0: the x lines (b = y, c = q, stride ny nt); axis 1: the y lines
// (b = x, c = q, stride nt), with the dispersion term.
template <typename T>
XYLine<T> line_args(fcn_xy_ctx *ctx, void *field, int axis, double dz) {
    XYLine<T> a;
    a.field = (cx<T> *)field;
    a.nt = ctx->g.nt;
    a.width = ctx->g.nt;
    a.total = ctx->points();
    double s, dk, disp;
    if (axis == 0) {
        line_coefs(ctx, dz, dx_of(ctx), &s, &dk, &disp);
        dk = 0.0;
        disp = 0.0;
        a.invden = (const cx<T> *)ctx->tab_x;
        a.n = ctx->g.nx;
        a.batch = ctx->g.ny;
        a.pitch = (long long)ctx->g.ny * ctx->g.nt;
        a.bstride = ctx->g.nt;
    } else {
        line_coefs(ctx, dz, dy_of(ctx), &s, &dk, &disp);
        a.invden = (const cx<T> *)ctx->tab_y;
        a.n = ctx->g.ny;
        a.batch = ctx->g.nx;
        a.pitch = ctx->g.nt;
        a.bstride = (long long)ctx->g.ny * ctx->g.nt;
    }
    a.s = T(s);
    a.dk = T(dk);
    a.s64 = s;
    a.dk64 = dk;
    a.disp = disp;
    a.variant = ctx->line_var;
    return a;
}

// Records an event pair around one launch when profiling is on.
template <typename F>
cudaError_t timed(fcn_xy_ctx *ctx, int kind, cudaStream_t st, F &&launch) {
    if (!ctx->profiling) return launch();
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
    cudaEventRecord(e0, st);
    e = launch();
    cudaEventRecord(e1, st);
    ctx->prof_events.push_back({kind, {e0, e1}});
    return e;
}

void profile_collect(fcn_xy_ctx *ctx) {
    for (auto &pe : ctx->prof_events) {
        float ms = 0.f;
        if (cudaEventSynchronize(pe.second.second) == cudaSuccess &&
            cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) {
            ctx->prof_ms[pe.first] += ms;
            ctx->prof_n[pe.first] += 1;
        }
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    ctx->prof_events.clear();
}

// Pivot tables of both axes for dz, rebuilt in place when dz changes (in
// stream order, after the launches that read the old tables).  Captured
// graphs read these buffers, so a rebuild drops them.
template <typename T>
int ensure_tables(fcn_xy_ctx *ctx, double dz) {
    if (ctx->tab_x && ctx->tab_dz == bits(dz)) return FCN_OK;
    if (!ctx->graphs.empty()) {
        CK(cudaStreamSynchronize(ctx->st), "sync before table rebuild");
        for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
        ctx->graphs.clear();
    }
    const int nq = ctx->g.nt / 2 + 1;
    if (!ctx->tab_x) {
        const size_t per = sizeof(cx<T>) * (sizeof(T) == 4 ? 2 : 1);   // FP32: two-float entries
        CK(cudaMalloc(&ctx->tab_x, per * (size_t)ctx->g.nx * nq), "x pivot table");
        CK(cudaMalloc(&ctx->tab_y, per * (size_t)ctx->g.ny * nq), "y pivot table");
    }
    double s, dk, disp;
    line_coefs(ctx, dz, dx_of(ctx), &s, &dk, &disp);
    CK(launch_xy_table<T>(ctx->g.nx, ctx->g.nt, s, 0.0, (cx<T> *)ctx->tab_x, ctx->st), "x pivot kernel");
    line_coefs(ctx, dz, dy_of(ctx), &s, &dk, &disp);
    CK(launch_xy_table<T>(ctx->g.ny, ctx->g.nt, s, dk, (cx<T> *)ctx->tab_y, ctx->st), "y pivot kernel");
    ctx->tab_dz = bits(dz);
    return FCN_OK;
}

// Variant timing per (precision, nx, ny, nt, K = 8 or not), process-wide:
// every row variant (FP32, K = 8) and line variant, three interleaved rounds
// of a few launches on a scratch copy of the field, the best round counting.
std::map<std::tuple<int, int, int, int, bool>, std::pair<int, int>> g_xy_tune;

template <typename F>
int time_launches(fcn_xy_ctx *ctx, F &&launch, float *ms_out) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    for (int i = 0; i < 2; ++i) CK(launch(), "tuning launch");
    cudaEventRecord(e0, ctx->st);
    for (int i = 0; i < 6; ++i) CK(launch(), "tuning launch");
    cudaEventRecord(e1, ctx->st);
    CK(cudaEventSynchronize(e1), "tuning sync");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = ms;
    return FCN_OK;
}

template <typename T>
int ensure_tuned(fcn_xy_ctx *ctx, double dz) {
    if (ctx->tuned) return FCN_OK;
    std::lock_guard<std::mutex> lk(g_xy_mu);
    auto key = std::make_tuple(ctx->prec, ctx->g.nx, ctx->g.ny, ctx->g.nt, ctx->p.K == 8);
    auto it = g_xy_tune.find(key);
    const bool need = (ctx->force_row < 0 || ctx->force_line < 0) && it == g_xy_tune.end();
    if (need) {
        const size_t bytes = csize(ctx->prec) * (size_t)ctx->points();
        void *scratch = nullptr;
        CK(cudaMalloc(&scratch, bytes), "tuning scratch");
        struct Free {
            void *p;
            ~Free() { cudaFree(p); }
        } guard{scratch};
        CK(cudaMemcpyAsync(scratch, ctx->field, bytes, cudaMemcpyDeviceToDevice, ctx->st), "tuning copy");
        const int nrv = (sizeof(T) == 4 && ctx->p.K == 8) ? kRowVariants : 1;
        std::vector<float> tr(nrv, 1e30f), tl(kXYVariants, 1e30f);
        for (int round = 0; round < 3; ++round) {
            for (int v = 0; v < nrv; ++v) {
                RowArgs<T> a = row_args<T>(ctx, scratch, OPS_MID, dz);
                a.variant = v;
                float ms;
                int rc = time_launches(ctx, [&] { return launch_rows<T>(a, ctx->g.nt, ctx->st); }, &ms);
                if (rc) return rc;
                tr[v] = std::min(tr[v], ms);
            }
            for (int v = 0; v < kXYVariants; ++v) {
                float ms0, ms1;
                XYLine<T> ax = line_args<T>(ctx, scratch, 0, dz), ay = line_args<T>(ctx, scratch, 1, dz);
                ax.variant = ay.variant = v;
                int rc = time_launches(ctx, [&] { return launch_xy_line<T>(ax, ctx->st); }, &ms0);
                if (!rc) rc = time_launches(ctx, [&] { return launch_xy_line<T>(ay, ctx->st); }, &ms1);
                if (rc) return rc;
                tl[v] = std::min(tl[v], ms0 + ms1);
            }
        }
        CK(cudaStreamSynchronize(ctx->st), "tuning sync");
        const int br = int(std::min_element(tr.begin(), tr.end()) - tr.begin());
        const int bl = int(std::min_element(tl.begin(), tl.end()) - tl.begin());
        it = g_xy_tune.emplace(key, std::make_pair(br, bl)).first;
    }
    ctx->row_var = ctx->force_row >= 0 ? ctx->force_row : it->second.first;
    ctx->line_var = ctx->force_line >= 0 ? ctx->force_line : it->second.second;
    ctx->tuned = true;
    return FCN_OK;
}

template <typename T>
cudaError_t launch_lines(fcn_xy_ctx *ctx, double dz, cudaStream_t st) {
    cudaError_t e = timed(ctx, FCN_XY_PROF_LINE_X, st,
                          [&] { return launch_xy_line<T>(line_args<T>(ctx, ctx->field, 0, dz), st); });
    if (e != cudaSuccess) return e;
    return timed(ctx, FCN_XY_PROF_LINE_Y, st,
                 [&] { return launch_xy_line<T>(line_args<T>(ctx, ctx->field, 1, dz), st); });
}

template <typename T>
cudaError_t launch_rows_op(fcn_xy_ctx *ctx, int ops, int kind, double dz, cudaStream_t st) {
    return timed(ctx, kind, st, [&] { return launch_rows<T>(row_args<T>(ctx, ctx->field, ops, dz), ctx->g.nt, st); });
}

// k (x lines, y lines, middle row stage) steps
template <typename T>
cudaError_t launch_mids(fcn_xy_ctx *ctx, double dz, int k, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < k && e == cudaSuccess; ++i) {
        e = launch_lines<T>(ctx, dz, st);
        if (e == cudaSuccess) e = launch_rows_op<T>(ctx, OPS_MID, FCN_XY_PROF_ROW_MID, dz, st);
    }
    return e;
}

template <typename T>
int run_mid8(fcn_xy_ctx *ctx, double dz, bool use_graph) {
    if (!use_graph || ctx->profiling) {
        CK(launch_mids<T>(ctx, dz, 8, ctx->st), "kernel launch");
        return FCN_OK;
    }
    auto it = ctx->graphs.find(bits(dz));
    if (it == ctx->graphs.end()) {
        cudaGraph_t gr = nullptr;
        CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t le = launch_mids<T>(ctx, dz, 8, ctx->cap);
        cudaError_t ce = cudaStreamEndCapture(ctx->cap, &gr);
        if (le != cudaSuccess) { if (gr) cudaGraphDestroy(gr); return cuda_fail(ctx, le, "captured launch"); }
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "end capture");
        cudaGraphExec_t ex = nullptr;
        cudaError_t ie = cudaGraphInstantiate(&ex, gr, 0);
        cudaGraphDestroy(gr);
        if (ie != cudaSuccess) return cuda_fail(ctx, ie, "graph instantiate");
        it = ctx->graphs.emplace(bits(dz), ex).first;
    }
    CK(cudaGraphLaunch(it->second, ctx->st), "graph launch");
    return FCN_OK;
}

template <typename T>
int step_impl(fcn_xy_ctx *ctx, double dz, int64_t n, bool use_graph) {
    if (!(dz > 0) || !std::isfinite(dz)) return fail(ctx, FCN_ERR_ARG, "dz must be > 0 and finite");
    if (n < 0) return fail(ctx, FCN_ERR_ARG, "n must be >= 0");
    if (!ctx->has_field) return fail(ctx, FCN_ERR_STATE, "fcn_xy_set_field has not been called");
    if (n == 0) return FCN_OK;
    int rc = ensure_tables<T>(ctx, dz);
    if (!rc) rc = ensure_tuned<T>(ctx, dz);
    if (rc) return rc;
    CK(launch_rows_op<T>(ctx, OPS_HEAD, FCN_XY_PROF_ROW_HEAD, dz, ctx->st), "head row stage");
    int64_t rem = n - 1;
    while (rem >= 8) {
        rc = run_mid8<T>(ctx, dz, use_graph);
        if (rc) return rc;
        rem -= 8;
    }
    CK(launch_mids<T>(ctx, dz, (int)rem, ctx->st), "middle steps");
    CK(launch_lines<T>(ctx, dz, ctx->st), "line stage");
    CK(launch_rows_op<T>(ctx, OPS_TAIL, FCN_XY_PROF_ROW_TAIL, dz, ctx->st), "tail row stage");
    ctx->z += dz * double(n);
    ctx->steps += n;
    return FCN_OK;
}

template <typename T>
int diag_impl(fcn_xy_ctx *ctx, fcn_diag *out) {
    RowArgs<T> a = row_args<T>(ctx, ctx->field, OP_STATS | OP_FFT | OP_SPEC | OP_NOSTORE, 0.0);
    a.variant = 0;
    CK(launch_rows<T>(a, ctx->g.nt, ctx->st), "diagnostics row pass");
    const int axis = ((ctx->g.nx - 1) / 2) * ctx->g.ny + (ctx->g.ny - 1) / 2;
    CK(launch_reduce_stats_flat(ctx->stats, (int)ctx->rows(), axis, ctx->red, ctx->st), "diagnostics reduction");
    CK(cudaMemcpyAsync(ctx->host_red, ctx->red, sizeof(double) * 8, cudaMemcpyDeviceToHost, ctx->st),
       "diagnostics copy");
    CK(cudaStreamSynchronize(ctx->st), "diagnostics sync");
    const double *r = ctx->host_red;
    double k0, dtau, domega;
    hostx::consts(ctx->rg, ctx->p, &k0, &dtau, &domega);
    std::memset(out, 0, sizeof(*out));
    out->z = ctx->z;
    out->energy = dx_of(ctx) * dy_of(ctx) * dtau * r[0];
    out->peak_intensity = r[1];
    out->peak_rho = r[2] * ctx->p.rho_nt;
    out->onaxis_peak = r[3];
    if (r[4] > 0) {
        const double mean = r[5] / r[4];
        const double var = r[6] / r[4] - mean * mean;
        out->spectral_rms = var > 0 ? std::sqrt(var) * domega : 0.0;
    }
    out->steps = ctx->steps;
    out->nonfinite = (r[7] > 0 || !std::isfinite(r[0])) ? 1 : 0;
    return out->nonfinite ? fail(ctx, FCN_ERR_NONFINITE, "field holds NaN or Inf") : FCN_OK;
}

int reset_state(fcn_xy_ctx *ctx) {
    CK(cudaMemsetAsync(ctx->stats, 0, sizeof(double) * NSTAT * (size_t)ctx->rows(), ctx->st), "reset stats");
    CK(cudaMemsetAsync(ctx->rho, 0, rsize(ctx->prec) * (size_t)ctx->points(), ctx->st), "reset rho");
    ctx->z = 0.0;
    ctx->steps = 0;
    ctx->has_field = true;
    return FCN_OK;
}

int ensure_stage(fcn_xy_ctx *ctx) {
    if (!ctx->stage) CK(cudaMalloc(&ctx->stage, 16 * (size_t)ctx->points()), "staging buffer");
    return FCN_OK;
}

}  // namespace

extern "C" {

int fcn_xy_create(const fcn_grid_xy *grid, const fcn_params *params, int32_t precision, void *stream,
                  fcn_xy_ctx **out) {
    if (!out) return fail(nullptr, FCN_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (!grid || !params) return fail(nullptr, FCN_ERR_ARG, "null grid or params");
    fcn_grid rg;
    rg.nr = 3;
    rg.nt = grid->nt;
    rg.r_max = 1.0;
    rg.t_window = grid->t_window;
    std::string why;
    int rc = hostx::check_params(precision, &rg, params, &why);
    if (rc) return fail(nullptr, rc, why);
    if (grid->nx < 3 || grid->ny < 3) return fail(nullptr, FCN_ERR_ARG, "nx and ny must be >= 3");
    if (grid->nx > 2048 || grid->ny > 2048)
        return fail(nullptr, FCN_ERR_UNSUPPORTED, "nx or ny > 2048 is not supported");
    if (!(grid->x_width > 0) || !std::isfinite(grid->x_width) || !(grid->y_width > 0) ||
        !std::isfinite(grid->y_width))
        return fail(nullptr, FCN_ERR_ARG, "x_width and y_width must be > 0");
    if ((int64_t)grid->nx * grid->ny > (int64_t)INT32_MAX / 2 ||
        (int64_t)grid->ny * grid->nt > (int64_t)INT32_MAX / 2)
        return fail(nullptr, FCN_ERR_UNSUPPORTED, "grid too large");
    fcn_xy_ctx *ctx = new fcn_xy_ctx;
    ctx->prec = precision;
    ctx->st = (cudaStream_t)stream;
    ctx->g = *grid;
    ctx->p = *params;
    ctx->rg = rg;
    const size_t np = (size_t)ctx->points();
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t b) {
        if (e == cudaSuccess) e = cudaMalloc(p, b);
    };
    alloc(&ctx->field, csize(precision) * np);
    alloc(&ctx->rho, rsize(precision) * np);
    alloc((void **)&ctx->stats, sizeof(double) * NSTAT * (size_t)ctx->rows());
    alloc((void **)&ctx->red, sizeof(double) * 16);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->host_red, sizeof(double) * 16);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        if (precision == FCN_FP64) {
            const cx<double> *tw;
            e = hostx::twiddles<double>(grid->nt, &tw);
            ctx->tw = tw;
            if (e == cudaSuccess) e = prepare_rows<double>(grid->nt);
        } else {
            const cx<float> *tw, *tw1 = nullptr;
            e = hostx::twiddles<float>(grid->nt, &tw);
            if (e == cudaSuccess && grid->nt >= 256) e = hostx::twiddles<float>(fft_tag(grid->nt, 1), &tw1);
            ctx->tw = tw;
            ctx->tw1 = tw1;
            if (e == cudaSuccess) e = prepare_rows<float>(grid->nt);
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->field, 0, csize(precision) * np, ctx->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->stats, 0, sizeof(double) * NSTAT * (size_t)ctx->rows(), ctx->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->rho, 0, rsize(precision) * np, ctx->st);
    if (e != cudaSuccess) {
        const int code = (e == cudaErrorMemoryAllocation) ? FCN_ERR_NOMEM : FCN_ERR_CUDA;
        fail(nullptr, code, std::string("context setup: ") + cudaGetErrorString(e));
        fcn_xy_destroy(ctx);
        return code;
    }
    *out = ctx;
    return FCN_OK;
}

void fcn_xy_destroy(fcn_xy_ctx *ctx) {
    if (!ctx) return;
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    cudaDeviceSynchronize();
    for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
    profile_collect(ctx);
    cudaFree(ctx->field);
    cudaFree(ctx->rho);
    cudaFree(ctx->stage);
    cudaFree(ctx->stats);
    cudaFree(ctx->red);
    cudaFree(ctx->tab_x);
    cudaFree(ctx->tab_y);
    if (ctx->host_red) cudaFreeHost(ctx->host_red);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    delete ctx;
}

const char *fcn_xy_last_error(const fcn_xy_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_xy_create_error.c_str();
}

int fcn_xy_set_field(fcn_xy_ctx *ctx, const double *host) {
    if (!ctx || !host) return fail(ctx, FCN_ERR_ARG, "null context or buffer");
    const size_t np = (size_t)ctx->points();
    if (ctx->prec == FCN_FP64) {
        CK(cudaMemcpyAsync(ctx->field, host, 16 * np, cudaMemcpyHostToDevice, ctx->st), "H2D field");
    } else {
        int rc = ensure_stage(ctx);
        if (rc) return rc;
        CK(cudaMemcpyAsync(ctx->stage, host, 16 * np, cudaMemcpyHostToDevice, ctx->st), "H2D field");
        CK(launch_narrow<float>((const double *)ctx->stage, (cx<float> *)ctx->field, (int64_t)np, ctx->st), "narrow");
    }
    return reset_state(ctx);
}

int fcn_xy_get_field(fcn_xy_ctx *ctx, double *host) {
    if (!ctx || !host) return fail(ctx, FCN_ERR_ARG, "null context or buffer");
    const size_t np = (size_t)ctx->points();
    if (ctx->prec == FCN_FP64) {
        CK(cudaMemcpyAsync(host, ctx->field, 16 * np, cudaMemcpyDeviceToHost, ctx->st), "D2H field");
    } else {
        int rc = ensure_stage(ctx);
        if (rc) return rc;
        CK(launch_widen<float>((const cx<float> *)ctx->field, (double *)ctx->stage, (int64_t)np, ctx->st), "widen");
        CK(cudaMemcpyAsync(host, ctx->stage, 16 * np, cudaMemcpyDeviceToHost, ctx->st), "D2H field");
    }
    CK(cudaStreamSynchronize(ctx->st), "sync");
    return FCN_OK;
}

int fcn_xy_set_field_c64(fcn_xy_ctx *ctx, const float *host) {
    if (!ctx || !host) return fail(ctx, FCN_ERR_ARG, "null context or buffer");
    const size_t np = (size_t)ctx->points();
    if (ctx->prec == FCN_FP32_MIXED) {
        CK(cudaMemcpyAsync(ctx->field, host, 8 * np, cudaMemcpyHostToDevice, ctx->st), "H2D field");
    } else {
        int rc = ensure_stage(ctx);
        if (rc) return rc;
        CK(cudaMemcpyAsync(ctx->stage, host, 8 * np, cudaMemcpyHostToDevice, ctx->st), "H2D field");
        CK(launch_widen<float>((const cx<float> *)ctx->stage, (double *)ctx->field, (int64_t)np, ctx->st), "widen");
    }
    return reset_state(ctx);
}

int fcn_xy_get_field_c64(fcn_xy_ctx *ctx, float *host) {
    if (!ctx || !host) return fail(ctx, FCN_ERR_ARG, "null context or buffer");
    const size_t np = (size_t)ctx->points();
    if (ctx->prec == FCN_FP32_MIXED) {
        CK(cudaMemcpyAsync(host, ctx->field, 8 * np, cudaMemcpyDeviceToHost, ctx->st), "D2H field");
    } else {
        int rc = ensure_stage(ctx);
        if (rc) return rc;
        CK(launch_narrow<float>((const double *)ctx->field, (cx<float> *)ctx->stage, (int64_t)np, ctx->st), "narrow");
        CK(cudaMemcpyAsync(host, ctx->stage, 8 * np, cudaMemcpyDeviceToHost, ctx->st), "D2H field");
    }
    CK(cudaStreamSynchronize(ctx->st), "sync");
    return FCN_OK;
}

int fcn_xy_set_field_device(fcn_xy_ctx *ctx, const void *dev) {
    if (!ctx || !dev) return fail(ctx, FCN_ERR_ARG, "null context or buffer");
    const size_t bytes = (ctx->prec == FCN_FP64 ? 16 : 8) * (size_t)ctx->points();
    CK(cudaMemcpyAsync(ctx->field, dev, bytes, cudaMemcpyDeviceToDevice, ctx->st), "D2D field");
    return reset_state(ctx);
}

int fcn_xy_get_field_device(fcn_xy_ctx *ctx, void *dev) {
    if (!ctx || !dev) return fail(ctx, FCN_ERR_ARG, "null context or buffer");
    const size_t bytes = (ctx->prec == FCN_FP64 ? 16 : 8) * (size_t)ctx->points();
    CK(cudaMemcpyAsync(dev, ctx->field, bytes, cudaMemcpyDeviceToDevice, ctx->st), "D2D field");
    return FCN_OK;
}

int fcn_xy_get_rho(fcn_xy_ctx *ctx, double *host) {
    if (!ctx || !host) return fail(ctx, FCN_ERR_ARG, "null context or buffer");
    const size_t np = (size_t)ctx->points();
    if (ctx->prec == FCN_FP64) {
        CK(cudaMemcpyAsync(host, ctx->rho, 8 * np, cudaMemcpyDeviceToHost, ctx->st), "D2H rho");
    } else {
        int rc = ensure_stage(ctx);
        if (rc) return rc;
        CK(launch_widen_real<float>((const float *)ctx->rho, (double *)ctx->stage, (int64_t)np, ctx->st), "widen rho");
        CK(cudaMemcpyAsync(host, ctx->stage, 8 * np, cudaMemcpyDeviceToHost, ctx->st), "D2H rho");
    }
    CK(cudaStreamSynchronize(ctx->st), "sync");
    return FCN_OK;
}

int fcn_xy_step(fcn_xy_ctx *ctx, double dz, int64_t n) {
    if (!ctx) return FCN_ERR_ARG;
    return ctx->prec == FCN_FP64 ? step_impl<double>(ctx, dz, n, true) : step_impl<float>(ctx, dz, n, true);
}

int fcn_xy_step_nograph(fcn_xy_ctx *ctx, double dz, int64_t n) {
    if (!ctx) return FCN_ERR_ARG;
    return ctx->prec == FCN_FP64 ? step_impl<double>(ctx, dz, n, false) : step_impl<float>(ctx, dz, n, false);
}

int fcn_xy_get_diag(fcn_xy_ctx *ctx, fcn_diag *out) {
    if (!ctx || !out) return fail(ctx, FCN_ERR_ARG, "null context or output");
    if (!ctx->has_field) return fail(ctx, FCN_ERR_STATE, "fcn_xy_set_field has not been called");
    return ctx->prec == FCN_FP64 ? diag_impl<double>(ctx, out) : diag_impl<float>(ctx, out);
}

int fcn_xy_set_variants(fcn_xy_ctx *ctx, int32_t row_variant, int32_t line_variant) {
    if (!ctx) return FCN_ERR_ARG;
    if (row_variant < -1 || row_variant >= kRowVariants || line_variant < -1 || line_variant >= kXYVariants)
        return fail(ctx, FCN_ERR_ARG, "variant out of range");
    CK(cudaStreamSynchronize(ctx->st), "sync");
    ctx->force_row = row_variant;
    ctx->force_line = line_variant;
    ctx->tuned = false;
    for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
    ctx->graphs.clear();
    return FCN_OK;
}

int fcn_xy_get_variants(const fcn_xy_ctx *ctx, int32_t out[2]) {
    if (!ctx || !out) return FCN_ERR_ARG;
    out[0] = ctx->row_var;
    out[1] = ctx->line_var;
    return FCN_OK;
}

int fcn_xy_profile_enable(fcn_xy_ctx *ctx, int32_t on) {
    if (!ctx) return FCN_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->st), "profile sync");
    profile_collect(ctx);
    ctx->profiling = on != 0;
    return FCN_OK;
}

int fcn_xy_profile_read(fcn_xy_ctx *ctx, double *ms, int64_t *count, int32_t reset) {
    if (!ctx || !ms || !count) return FCN_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->st), "profile sync");
    profile_collect(ctx);
    for (int k = 0; k < FCN_XY_PROF_KINDS; ++k) {
        ms[k] = ctx->prof_ms[k];
        count[k] = ctx->prof_n[k];
        if (reset) {
            ctx->prof_ms[k] = 0;
            ctx->prof_n[k] = 0;
        }
    }
    return FCN_OK;
}

}  // extern "C"
