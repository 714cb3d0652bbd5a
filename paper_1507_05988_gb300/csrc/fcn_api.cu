// fcn_api.cu -- C-ABI of the GB300 FCN z-step library (declared in
// include/fcn.h).  Host-side orchestration only: argument checks, physical
// constants, device buffers, the pivot-table cache, CUDA-graph capture of
// the z-loop and the step-doubling controller.  Every arithmetic step of
// the z-step runs in the kernels of row_kernel.cu, col_kernel.cu and
// reduce.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <tuple>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fcn.h"
#include "fcn_device.cuh"
#include "fcn_host.h"

using namespace fcn;

namespace {

// CODATA 2018 (SI)
constexpr double kC = 299792458.0;
constexpr double kHbar = 1.054571817e-34;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMe = 9.1093837015e-31;
constexpr double kQe = 1.602176634e-19;
constexpr double kPi = 3.14159265358979323846;
// Intensity scale of the nonlinear stage: a power of two, so Ihat = I/I_s is
// exact; 2^53 W/m^2 ~ 9e15 keeps Ihat^K inside FP32 range for I up to ~5e20.
constexpr double kIs = 9007199254740992.0;

std::string g_create_error = "no error";
std::mutex g_mu;

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

int check_grid_params(int prec, const fcn_grid *g, const fcn_params *p, std::string *why) {
    if (!g || !p) { *why = "null grid or params"; return FCN_ERR_ARG; }
    if (prec != FCN_FP64 && prec != FCN_FP32_MIXED) { *why = "unknown precision"; return FCN_ERR_ARG; }
    if (!is_pow2(g->nt) || g->nt < 2) { *why = "nt must be a power of two >= 2"; return FCN_ERR_ARG; }
    if (g->nt > 8192) { *why = "nt > 8192 is not supported"; return FCN_ERR_UNSUPPORTED; }
    if (g->nr < 3) { *why = "nr must be >= 3"; return FCN_ERR_ARG; }
    if (g->nr > 2048) { *why = "nr > 2048 is not supported"; return FCN_ERR_UNSUPPORTED; }
    if (!(g->r_max > 0) || !std::isfinite(g->r_max)) { *why = "r_max must be > 0"; return FCN_ERR_ARG; }
    if (!(g->t_window > 0) || !std::isfinite(g->t_window)) { *why = "t_window must be > 0"; return FCN_ERR_ARG; }
    if (!(p->lambda0 > 0) || !(p->n0 > 0)) { *why = "lambda0 and n0 must be > 0"; return FCN_ERR_ARG; }
    if (p->K < 1 || p->K > 16) { *why = "K must be in 1..16"; return FCN_ERR_ARG; }
    if (p->flags & ~(63u | FCN_EXACT_DISPERSION)) { *why = "unknown physics flag"; return FCN_ERR_ARG; }
    if (!(p->sigma_k >= 0) || !(p->rho_nt >= 0) || !std::isfinite(p->k2)) {
        *why = "sigma_k, rho_nt must be >= 0 and k2 finite"; return FCN_ERR_ARG;
    }
    for (int j = 0; j < 4; ++j)
        if (!std::isfinite(p->n2j[j])) { *why = "n2j must be finite"; return FCN_ERR_ARG; }
    return FCN_OK;
}

// Derived constants of one pulse (host, FP64).
struct Consts {
    double k0, omega0, rho_c, beta_k, dr, dtau, domega;
};

Consts derive(const fcn_grid &g, const fcn_params &p) {
    Consts c;
    c.k0 = 2.0 * kPi * p.n0 / p.lambda0;
    c.omega0 = 2.0 * kPi * kC / p.lambda0;
    c.rho_c = kEps0 * kMe * c.omega0 * c.omega0 / (kQe * kQe);
    c.beta_k = double(p.K) * kHbar * c.omega0 * p.sigma_k * p.rho_nt;
    c.dr = g.r_max / double(g.nr - 1);
    c.dtau = g.t_window / double(g.nt);
    c.domega = 2.0 * kPi / (double(g.nt) * c.dtau);
    return c;
}

template <typename T>
NLCoef<T> nl_coef(const fcn_grid &g, const fcn_params &p, double h) {
    const Consts c = derive(g, p);
    NLCoef<T> n;
    n.h = T(h);
    double isj = kIs;
    for (int j = 0; j < 4; ++j) {
        n.kerr[j] = T((c.k0 / p.n0) * p.n2j[j] * isj);
        isj *= kIs;
    }
    n.plasma = T(c.k0 / (2.0 * p.n0 * p.n0 * c.rho_c) * p.rho_nt);
    n.loss = T(0.5 * c.beta_k * std::pow(kIs, p.K - 1));
    n.sdt = T(p.sigma_k * c.dtau * std::pow(kIs, p.K));
    n.inv_is = T(1.0 / kIs);
    n.inv_nt = T(1.0 / double(g.nt));
    n.rho_nt = T(p.rho_nt);
    n.K = p.K;
    n.nkerr = 1;
    for (int j = 0; j < 4; ++j)
        if (p.n2j[j] != 0.0) n.nkerr = j + 1;
    n.flags = p.flags;
    isj = kIs;
    for (int j = 0; j < 4; ++j) {
        n.hk[j] = (p.flags & FCN_KERR) ? T(h * (c.k0 / p.n0) * p.n2j[j] * isj) : T(0);
        isj *= kIs;
    }
    n.hplasma = (p.flags & FCN_PLASMA) ? T(h * (c.k0 / (2.0 * p.n0 * p.n0 * c.rho_c) * p.rho_nt)) : T(0);
    n.hloss = (p.flags & FCN_MPI) ? T(h * 0.5 * c.beta_k * std::pow(kIs, p.K - 1)) : T(0);
    n.sat = (p.flags & FCN_MPI_SAT) ? T(1) : T(0);
    const double sdt = p.sigma_k * c.dtau * std::pow(kIs, p.K);
    n.is_root = T(sdt > 0.0 ? std::pow(sdt, 1.0 / p.K) / kIs : 0.0);
    return n;
}

// s and dk of the CN system (delta_q = dk q^2 on its diagonal); with
// FCN_EXACT_DISPERSION dk = 0 and *disp receives the coefficient of the exact
// factor exp(2 i disp q^2) the column stage applies instead.
void cn_coefs(const fcn_grid &g, const fcn_params &p, double dz, double *s, double *dk,
              double *disp = nullptr) {
    const Consts c = derive(g, p);
    *s = (p.flags & FCN_DIFFRACTION) ? dz / (4.0 * c.k0 * c.dr * c.dr) : 0.0;
    const double d = (p.flags & FCN_DISPERSION) ? p.k2 * dz / 4.0 * c.domega * c.domega : 0.0;
    const bool exact = (p.flags & FCN_EXACT_DISPERSION) != 0;
    *dk = exact ? 0.0 : d;
    if (disp) *disp = exact ? d : 0.0;
}

// ---- process-wide constant tables (twiddles, radial ratios) ----
struct ConstTables {
    std::map<std::pair<int, int>, void *> tw;      // (prec, nt with FFT plan tag) -> twiddle blocks
    std::map<std::pair<int, int>, void *> lohi;    // (prec, nr) -> T[2*nr]
    std::map<int, double *> lohi64;                // nr -> double[2*nr]
};
ConstTables g_tables;

// ntp: Nt with the FFT plan in its high bits (fft_tag)
template <typename T>
cudaError_t get_twiddles(int ntp, const cx<T> **out) {
    const int prec = sizeof(T) == 8 ? FCN_FP64 : FCN_FP32_MIXED;
    const int nt = fft_nt(ntp);
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_pair(prec, ntp);
    auto it = g_tables.tw.find(key);
    if (it != g_tables.tw.end()) { *out = (const cx<T> *)it->second; return cudaSuccess; }
    // W^m = exp(-2 pi i m / nt); FP32 entries as two-float pairs (hi, lo):
    // hi the nearest float, lo the nearest float to the remainder, so that
    // hi + lo carries the twiddle to ~1e-15 in phase and modulus
    constexpr int PER = sizeof(T) == 4 ? 2 : 1;        // cx<T> values per entry
    std::vector<cx<T>> w((size_t)nt * PER);
    for (int m = 0; m < nt; ++m) {
        const long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)m /
                                (long double)nt;
        const long double c = cosl(ang), sn = sinl(ang);
        if constexpr (sizeof(T) == 4) {
            const float ch = float(c), sh = float(sn);
            w[2 * (size_t)m] = mk(ch, sh);
            w[2 * (size_t)m + 1] = mk(float(c - (long double)ch), float(sn - (long double)sh));
        } else {
            w[m] = mk(T(c), T(sn));
        }
    }
    // per-pass blocks (layout in fcn_device.cuh: tw_offset)
    const size_t n = std::max(1, tw_size(ntp));
    std::vector<cx<T>> h(n * PER, mk(T(0), T(0)));
    for (int p = 1; p < fft_npass(ntp); ++p) {
        const int R = fft_radix(ntp, p), NS = fft_ns(ntp, p), stride = nt / (NS * R);
        for (int r = 1; r < R; ++r)
            for (int k = 0; k < NS; ++k)
                for (int u = 0; u < PER; ++u)
                    h[((size_t)tw_offset(ntp, p) + (r - 1) * NS + k) * PER + u] =
                        w[(size_t)(r * k * stride) * PER + u];
    }
    void *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(cx<T>) * n * PER);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(d, h.data(), sizeof(cx<T>) * n * PER, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(d); return e; }
    g_tables.tw[key] = d;
    *out = (const cx<T> *)d;
    return cudaSuccess;
}

// lo_j = 1 - 1/(2j), hi_j = 1 + 1/(2j) (0 at j = 0), same FP64 expression as
// the coefficients of Eq. (matrix1).
template <typename T>
cudaError_t get_lohi(int nr, const T **lo, const T **hi, const double **lo64, const double **hi64) {
    const int prec = sizeof(T) == 8 ? FCN_FP64 : FCN_FP32_MIXED;
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_pair(prec, nr);
    std::vector<double> h(2 * nr, 0.0);
    for (int j = 1; j < nr; ++j) {
        h[j] = 1.0 - 1.0 / (2.0 * j);
        h[nr + j] = 1.0 + 1.0 / (2.0 * j);
    }
    cudaError_t e;
    auto it = g_tables.lohi.find(key);
    if (it == g_tables.lohi.end()) {
        std::vector<T> ht(2 * nr);
        for (int i = 0; i < 2 * nr; ++i) ht[i] = T(h[i]);
        void *d = nullptr;
        if ((e = cudaMalloc(&d, sizeof(T) * 2 * nr)) != cudaSuccess) return e;
        if ((e = cudaMemcpy(d, ht.data(), sizeof(T) * 2 * nr, cudaMemcpyHostToDevice)) != cudaSuccess) {
            cudaFree(d);
            return e;
        }
        it = g_tables.lohi.emplace(key, d).first;
    }
    auto it64 = g_tables.lohi64.find(nr);
    if (it64 == g_tables.lohi64.end()) {
        double *d = nullptr;
        if ((e = cudaMalloc(&d, sizeof(double) * 2 * nr)) != cudaSuccess) return e;
        if ((e = cudaMemcpy(d, h.data(), sizeof(double) * 2 * nr, cudaMemcpyHostToDevice)) != cudaSuccess) {
            cudaFree(d);
            return e;
        }
        it64 = g_tables.lohi64.emplace(nr, d).first;
    }
    *lo = (const T *)it->second;
    *hi = (const T *)it->second + nr;
    *lo64 = it64->second;
    *hi64 = it64->second + nr;
    return cudaSuccess;
}

size_t csize(int prec) { return prec == FCN_FP64 ? 16 : 8; }
size_t rsize(int prec) { return prec == FCN_FP64 ? 8 : 4; }

}  // namespace

// Host helpers shared with the Cartesian-grid API (xy_api.cu; fcn_host.h).
namespace fcn {
namespace hostx {
int check_params(int prec, const fcn_grid *g, const fcn_params *p, std::string *why) {
    return check_grid_params(prec, g, p, why);
}
template <typename T>
NLCoef<T> nl(const fcn_grid &g, const fcn_params &p, double h) {
    return nl_coef<T>(g, p, h);
}
template NLCoef<float> nl<float>(const fcn_grid &, const fcn_params &, double);
template NLCoef<double> nl<double>(const fcn_grid &, const fcn_params &, double);
template <typename T>
cudaError_t twiddles(int ntp, const cx<T> **out) {
    return get_twiddles<T>(ntp, out);
}
template cudaError_t twiddles<float>(int, const cx<float> **);
template cudaError_t twiddles<double>(int, const cx<double> **);
void consts(const fcn_grid &g, const fcn_params &p, double *k0, double *dtau, double *domega) {
    const Consts c = derive(g, p);
    *k0 = c.k0;
    *dtau = c.dtau;
    *domega = c.domega;
}
void cn_coefs(const fcn_grid &g, const fcn_params &p, double dz, double *s, double *dk,
              double *disp) {
    ::cn_coefs(g, p, dz, s, dk, disp);
}
}  // namespace hostx
}  // namespace fcn


// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

struct Pulse {
    fcn_grid g;
    fcn_params p;
    void *field = nullptr;     // current state (time domain between calls)
    void *work1 = nullptr;     // adaptive: one-step result
    void *work2 = nullptr;     // adaptive: two-half-step result
    void *rho = nullptr;       // T[nr*nt]
    double *stats = nullptr;   // [nr*NSTAT]
    double *red = nullptr;     // [16] reduction outputs
    double *rows = nullptr;    // [2*nr] row partials
    double *stage = nullptr;   // double staging [2*nr*nt] for host transfers
    int *err = nullptr;        // [1] set by a kernel whose bounded wait gave up
    const void *tw = nullptr;
    const void *tw1 = nullptr;   // twiddles of FFT plan 1 (FP32, Nt >= 256), or null
    const void *lo = nullptr, *hi = nullptr;
    const double *lo64 = nullptr, *hi64 = nullptr;
    double z = 0.0, dz_next = 0.0;
    int64_t steps = 0, rejected = 0;
    bool has_field = false;
    int row_var = 0, col_var = 0;   // kernel variants in use
    bool tuned = false;
    int64_t points() const { return (int64_t)g.nr * g.nt; }
};

struct TableKey {
    int nr, nt;
    uint64_t s, dk;   // bit patterns of s and the delta coefficient
    bool operator<(const TableKey &o) const {
        if (nr != o.nr) return nr < o.nr;
        if (nt != o.nt) return nt < o.nt;
        if (s != o.s) return s < o.s;
        return dk < o.dk;
    }
};

struct TableEntry {
    void *ptr;
    uint64_t dz;      // dz bits the table was built for (graphs keyed by dz)
    uint64_t stamp;   // last use
    size_t bytes;     // allocation size
};

constexpr int kMaxBranches = 8;

struct GraphKey {
    int kind;        // 0 head, 1 mid x8, 2 mid x1, 3 tail; + 4: captured with timing events
    uint64_t dz;
    bool operator<(const GraphKey &o) const { return kind != o.kind ? kind < o.kind : dz < o.dz; }
};

struct fcn_ctx {
    int prec = FCN_FP64;
    cudaStream_t st = nullptr;        // user stream (launch target)
    cudaStream_t cap = nullptr;       // internal stream used for graph capture
    // graph branches: the pulse groups (pairs or single pulses) of a captured
    // block are independent chains; with branches > 1 they are captured on
    // that many forked streams so that the GPU overlaps them
    int branches = 1;
    // multi-pulse row launches: 0 one launch per pulse; 1 per z-step the
    // column launches of all groups, then one row launch over all pulses;
    // 2 per group (a paired column launch's two pulses) one row launch
    int multi_mode = 2;
    cudaStream_t bst[kMaxBranches] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kMaxBranches] = {};
    // pivot tables built off the launch stream (adaptive steps need two new
    // tables per attempt, for dz and dz/2): streams, "launch stream reached
    // here" events and "table ready" events
    cudaStream_t tside[2] = {};
    cudaEvent_t tbefore[2] = {}, tready[2] = {};
    std::vector<Pulse> pulses;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::map<TableKey, TableEntry> tables;   // shared pivot tables
    uint64_t table_clock = 0;
    std::string err = "no error";
    double *host_red = nullptr;       // pinned [16]
    // kernel timing (fcn_profile_enable): one event pair per launch, by kind
    // kernel timing: 0 off, 1 direct launches with an event pair each, 2
    // graphs captured with an event record node before and after each kernel
    int profiling = 0;
    using EvList = std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>>;
    EvList prof_events;
    std::map<GraphKey, EvList> graph_events;   // the events of each timed graph
    EvList *cap_events = nullptr;              // set while a timed graph is captured
    double prof_ms[FCN_PROF_KINDS] = {0};
    int64_t prof_n[FCN_PROF_KINDS] = {0};
    float *mlp = nullptr;             // device FP32 master weights (FCN_MLP_NPARAM)
    bool has_mlp = false;
    unsigned char *mlp_io = nullptr;  // controller output: 8 doubles
    unsigned char *batch_io = nullptr;  // the same per pulse of an adaptive batch (64 B each)
    size_t batch_cap = 0;               // pulses batch_io and host_ctl hold
    double *host_ctl = nullptr;         // pinned, 16 doubles per pulse of an adaptive batch
    float *log_buf = nullptr;         // caller-owned host log of adaptive attempts
    int64_t log_cap = 0, log_n = 0;
    int force_row = -1, force_col = -1;   // -1: autotune; else forced variant
    // paired column launches for pulses sharing a grid and table (FP32):
    // mode -1 decides by timing, 0 off, 1 on; pairs is the decision (-1 open)
    int pair_mode = -1, pairs = -1;
    // the sequential column kernel over all pulses in one launch (equal
    // grids, one pivot table): mode -1 decide by timing, 0 off, 1 on;
    // seq_all is the decision (-1 before the first step), seq_shape the
    // ring shape the tuner chose for it
    int seq_mode = -1, seq_all = -1, seq_shape = 0;
    // batched work lists (FP32, K = 8, several pulses): one launch per stage
    bool batched = false;
    int2 *row_items = nullptr;
    int nrow_items = 0;
    int4 *col_items = nullptr;
    int ncol_items = 0;
    unsigned *counter = nullptr;
    size_t row_smem = 0;
    int row_grid = 0, col_grid = 0;
    std::map<uint64_t, std::pair<void *, void *>> batch_args;   // dz -> (RowArgs[], ColArgs[])
};

namespace {

int fail(fcn_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(fcn_ctx *c, cudaError_t e, const char *what) {
    return fail(c, FCN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

uint64_t dz_key(double dz) {
    uint64_t k;
    std::memcpy(&k, &dz, sizeof k);
    return k;
}

// Pivot tables are shared by every pulse of the context whose (Nr, Nt, s,
// delta coefficient) match -- identical grids and physics at the same dz --
// so a batch of equal pulses streams one table (L2-resident) instead of one
// per pulse.  Least-recently used tables beyond 2 per pulse + 8 are freed,
// together with the graphs and batch arguments captured with them.
// A context table allocation holds the pivots ([nr][nt/2+1] complex) and,
// from this byte offset on, the nr CnCoef rows of the staged column kernels.
template <typename T>
size_t coef_offset(int nr, int nt) {
    const size_t b = sizeof(cx<T>) * (size_t)nr * (size_t)table_pitch(nt);
    return (b + 255) / 256 * 256;
}
// then, in FP32, the per-column constants (ColConst, table_pitch entries)
template <typename T>
size_t cc_offset(int nr, int nt) {
    const size_t b = coef_offset<T>(nr, nt) + sizeof(CnCoef<T>) * (size_t)nr;
    return (b + 255) / 256 * 256;
}
template <typename T>
size_t table_bytes(int nr, int nt) {
    return sizeof(T) == 4 ? cc_offset<T>(nr, nt) + sizeof(ColConst) * (size_t)table_pitch(nt)
                          : coef_offset<T>(nr, nt) + sizeof(CnCoef<T>) * (size_t)nr;
}

void drop_graphs(fcn_ctx *ctx, bool all, uint64_t dz);

// The pivot table of (grid, dz), built on first use.  side = -1 builds it on
// the launch stream; side = 0 or 1 builds it on a side stream (after all
// work already queued on the launch stream, which may still read an evicted
// buffer) and sets *ready to an event that the launch stream must wait on
// before the table is read (null when the table was cached).
template <typename T>
int ensure_table(fcn_ctx *ctx, Pulse &pu, double dz, const cx<T> **out, int side = -1,
                 cudaEvent_t *ready = nullptr) {
    if (ready) *ready = nullptr;
    TableKey key;
    key.nr = pu.g.nr;
    key.nt = pu.g.nt;
    double s, dk;
    cn_coefs(pu.g, pu.p, dz, &s, &dk);
    key.s = dz_key(s);
    key.dk = dz_key(dk);
    auto it = ctx->tables.find(key);
    if (it != ctx->tables.end()) {
        it->second.stamp = ++ctx->table_clock;
        *out = (const cx<T> *)it->second.ptr;
        return FCN_OK;
    }
    const size_t need = table_bytes<T>(pu.g.nr, pu.g.nt);
    void *d = nullptr;
    const size_t cap = 2 * ctx->pulses.size() + 8;
    if (ctx->tables.size() >= cap) {
        auto old = ctx->tables.begin();
        for (auto t = ctx->tables.begin(); t != ctx->tables.end(); ++t)
            if (t->second.stamp < old->second.stamp) old = t;
        const uint64_t odz = old->second.dz;
        bool dropped = false;
        for (int kind = 0; kind < 8; ++kind) dropped |= ctx->graphs.count(GraphKey{kind, odz}) > 0;
        dropped |= ctx->batch_args.count(odz) > 0;
        if (dropped) {
            // graphs and argument arrays that refer to the table go with it
            CK(cudaStreamSynchronize(ctx->st), "sync before table eviction");
            drop_graphs(ctx, false, odz);
            auto ba = ctx->batch_args.find(odz);
            if (ba != ctx->batch_args.end()) {
                cudaFree(ba->second.first);
                cudaFree(ba->second.second);
                ctx->batch_args.erase(ba);
            }
        }
        if (old->second.bytes == need) {
            // reused in stream order: the kernels that read the old table run
            // on this stream before the ones that rebuild it (an adaptive run
            // replaces tables at every new dz, so no allocation per attempt)
            d = old->second.ptr;
        } else {
            cudaFree(old->second.ptr);
        }
        ctx->tables.erase(old);
    }
    if (!d) CK(cudaMalloc(&d, need), "pivot table allocation");
    TableArgs ta;
    ta.nr = pu.g.nr;
    ta.nt = pu.g.nt;
    ta.s = s;
    ta.dk = dk;
    ta.lo = pu.lo64;
    ta.hi = pu.hi64;
    ta.tp = table_pitch(pu.g.nt);
    ta.pivlim = ctx->prec == FCN_FP32_MIXED ? 1 : 0;
    if (sizeof(T) == 4) ta.cc = (ColConst *)((char *)d + cc_offset<T>(pu.g.nr, pu.g.nt));
    cudaStream_t bs = ctx->st;
    if (side >= 0) {
        if (!ctx->tside[side]) {
            CK(cudaStreamCreateWithFlags(&ctx->tside[side], cudaStreamNonBlocking), "table stream");
            CK(cudaEventCreateWithFlags(&ctx->tbefore[side], cudaEventDisableTiming), "table event");
            CK(cudaEventCreateWithFlags(&ctx->tready[side], cudaEventDisableTiming), "table event");
        }
        bs = ctx->tside[side];
        CK(cudaEventRecord(ctx->tbefore[side], ctx->st), "table event");
        CK(cudaStreamWaitEvent(bs, ctx->tbefore[side], 0), "table wait");
    }
    CnCoef<T> *coef = (CnCoef<T> *)((char *)d + coef_offset<T>(pu.g.nr, pu.g.nt));
    CK(launch_cn_coef<T>(ta, coef, bs), "row coefficient kernel");
    CK(launch_cn_table<T>(ta, (cx<T> *)d, bs), "pivot table kernel");
    if (side >= 0) {
        CK(cudaEventRecord(ctx->tready[side], bs), "table event");
        if (ready) *ready = ctx->tready[side];
        else CK(cudaStreamWaitEvent(ctx->st, ctx->tready[side], 0), "table wait");
    }
    ctx->tables[key] = TableEntry{d, dz_key(dz), ++ctx->table_clock, need};
    *out = (const cx<T> *)d;
    return FCN_OK;
}

template <typename T>
RowArgs<T> row_args(Pulse &pu, void *field, int ops, double dz) {
    RowArgs<T> a;
    a.field = (cx<T> *)field;
    a.tw = (const cx<T> *)pu.tw;
    a.tw1 = (const cx<T> *)pu.tw1;
    a.rho = (T *)pu.rho;
    a.stats = pu.stats;
    a.nr = pu.g.nr;
    a.nt = pu.g.nt;
    a.ops = ops;
    a.variant = pu.row_var;
    a.nl = nl_coef<T>(pu.g, pu.p, 0.5 * dz);
    a.err = pu.err;
    return a;
}

template <typename T>
ColArgs<T> col_args(Pulse &pu, void *field, const cx<T> *table, double dz) {
    ColArgs<T> a;
    a.field = (cx<T> *)field;
    a.invden = table;
    a.coef = (const CnCoef<T> *)((const char *)table + coef_offset<T>(pu.g.nr, pu.g.nt));
    a.lo = (const T *)pu.lo;
    a.hi = (const T *)pu.hi;
    a.nr = pu.g.nr;
    a.nt = pu.g.nt;
    double s, dk, disp;
    cn_coefs(pu.g, pu.p, dz, &s, &dk, &disp);
    a.s = T(s);
    a.dk = T(dk);
    a.s64 = s;
    a.dk64 = dk;
    a.disp = disp;
    a.variant = pu.col_var;
    a.tp = table_pitch(pu.g.nt);
    a.err = pu.err;
    a.pivlim = sizeof(T) == 4 ? 1 : 0;   // FP32 context tables hold deltas (ensure_table)
    if (sizeof(T) == 4) a.cc = (const ColConst *)((const char *)table + cc_offset<T>(pu.g.nr, pu.g.nt));
    return a;
}

// Records an event pair around one launch when profiling is on.
template <typename F>
cudaError_t timed(fcn_ctx *ctx, int kind, cudaStream_t st, F &&launch) {
    if (!ctx->profiling) return launch();
    if (ctx->profiling == 2) {
        // inside a capture the two records become event nodes of the graph
        if (!ctx->cap_events) return launch();
        cudaEvent_t e0, e1;
        cudaError_t e = cudaEventCreate(&e0);
        if (e != cudaSuccess) return e;
        if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
        ctx->cap_events->push_back({kind, {e0, e1}});
        // "external" records: event nodes of the graph, recorded at every
        // replay (a plain record inside a capture only orders the capture)
        if ((e = cudaEventRecordWithFlags(e0, st, cudaEventRecordExternal)) != cudaSuccess) return e;
        if ((e = launch()) != cudaSuccess) return e;
        return cudaEventRecordWithFlags(e1, st, cudaEventRecordExternal);
    }
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
    cudaEventRecord(e0, st);
    e = launch();
    cudaEventRecord(e1, st);
    ctx->prof_events.push_back({kind, {e0, e1}});
    return e;
}

void profile_collect(fcn_ctx *ctx) {
    for (auto &pe : ctx->prof_events) {
        float ms = 0.f;
        cudaEventSynchronize(pe.second.second);
        if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) {
            ctx->prof_ms[pe.first] += ms;
            ctx->prof_n[pe.first] += 1;
        }
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    ctx->prof_events.clear();
}

// Destroys the captured graphs (all, or those of one dz bit pattern) and the
// timing events that belong to them.
void drop_graphs(fcn_ctx *ctx, bool all, uint64_t dz) {
    for (auto it = ctx->graphs.begin(); it != ctx->graphs.end();) {
        if (!all && it->first.dz != dz) { ++it; continue; }
        cudaGraphExecDestroy(it->second);
        auto ev = ctx->graph_events.find(it->first);
        if (ev != ctx->graph_events.end()) {
            for (auto &pe : ev->second) {
                cudaEventDestroy(pe.second.first);
                cudaEventDestroy(pe.second.second);
            }
            ctx->graph_events.erase(ev);
        }
        it = ctx->graphs.erase(it);
    }
}

constexpr int OPS_HEAD = OP_NL | OP_FFT;
constexpr int OPS_MID = OP_IFFT | OP_NL | OP_NL2 | OP_FFT;
constexpr int OPS_TAIL = OP_IFFT | OP_NL | OP_RHO | OP_STATS;
// The closing launch of a state that is never kept (the one-step result of a
// step-doubling attempt, which only enters the error norm): no rho output and
// no statistics, so no u rows in shared memory either.
constexpr int OPS_TAIL_BARE = OP_IFFT | OP_NL;

// Launches `kind` for every pulse on stream st: 0 head, 1 eight (col, mid)
// pairs, 2 one (col, mid) pair, 3 (col, tail), 5 (col, bare tail).
// Device argument arrays of the batched kernels for this dz (built once).
template <typename T>
cudaError_t batch_args(fcn_ctx *ctx, double dz, const std::vector<const cx<T> *> &tabs,
                       const RowArgs<T> **ra, const ColArgs<T> **ca) {
    const uint64_t key = dz_key(dz);
    auto it = ctx->batch_args.find(key);
    if (it == ctx->batch_args.end()) {
        const size_t n = ctx->pulses.size();
        std::vector<RowArgs<T>> hr(n);
        std::vector<ColArgs<T>> hc(n);
        for (size_t i = 0; i < n; ++i) {
            hr[i] = row_args<T>(ctx->pulses[i], ctx->pulses[i].field, 0, dz);
            hc[i] = col_args<T>(ctx->pulses[i], ctx->pulses[i].field, tabs[i], dz);
        }
        void *dr = nullptr, *dc = nullptr;
        cudaError_t e = cudaMalloc(&dr, sizeof(RowArgs<T>) * n);
        if (e == cudaSuccess) e = cudaMalloc(&dc, sizeof(ColArgs<T>) * n);
        if (e == cudaSuccess) e = cudaMemcpy(dr, hr.data(), sizeof(RowArgs<T>) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dc, hc.data(), sizeof(ColArgs<T>) * n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(dr);
            cudaFree(dc);
            return e;
        }
        it = ctx->batch_args.emplace(key, std::make_pair(dr, dc)).first;
    }
    *ra = (const RowArgs<T> *)it->second.first;
    *ca = (const ColArgs<T> *)it->second.second;
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_block_batched(fcn_ctx *ctx, int kind, double dz, cudaStream_t st,
                                 const std::vector<const cx<T> *> &tabs) {
    if constexpr (sizeof(T) != 4) {
        return cudaErrorNotSupported;
    } else {
        const RowArgs<T> *ra;
        const ColArgs<T> *ca;
        cudaError_t e = batch_args<T>(ctx, dz, tabs, &ra, &ca);
        if (e != cudaSuccess) return e;
        auto rows = [&](int ops, int pk) {
            return timed(ctx, pk, st, [&] {
                return launch_rows_batch<T>(ra, ctx->row_items, ctx->nrow_items, ops, ctx->counter,
                                            ctx->row_smem, ctx->row_grid, st);
            });
        };
        auto col = [&] {
            return timed(ctx, FCN_PROF_COLUMN, st, [&] {
                return launch_cn_batch<T>(ca, ctx->col_items, ctx->ncol_items, ctx->counter,
                                          ctx->col_grid, st);
            });
        };
        if (kind == 0) {
            e = rows(OPS_HEAD, FCN_PROF_ROW_HEAD);
        } else if (kind == 1 || kind == 2) {
            const int reps = kind == 1 ? 8 : 1;
            for (int r = 0; r < reps && e == cudaSuccess; ++r) {
                e = col();
                if (e == cudaSuccess) e = rows(OPS_MID, FCN_PROF_ROW_MID);
            }
        } else {
            e = col();
            if (e == cudaSuccess) e = rows(kind == 5 ? OPS_TAIL_BARE : OPS_TAIL, FCN_PROF_ROW_TAIL);
        }
        return e;
    }
}

// Whether pulses i and i+1 take one paired column launch: pairing chosen,
// FP32, same grid and the same pivot table.
template <typename T>
bool pairable(const fcn_ctx *ctx, const std::vector<const cx<T> *> &tabs, size_t i) {
    if (sizeof(T) != 4 || ctx->pairs != 1 || i + 1 >= ctx->pulses.size()) return false;
    const Pulse &a = ctx->pulses[i], &b = ctx->pulses[i + 1];
    return a.g.nr == b.g.nr && a.g.nt == b.g.nt && tabs[i] == tabs[i + 1];
}

// Whether two pulses' row launches differ only in their field, rho and
// statistics pointers (same grid, twiddles, operations, variant and
// coefficients), so that one multi-pulse launch serves both.
template <typename T>
bool same_row_launch(const RowArgs<T> &a, const RowArgs<T> &b) {
    const NLCoef<T> &x = a.nl, &y = b.nl;
    bool same = a.nr == b.nr && a.nt == b.nt && a.tw == b.tw && a.ops == b.ops && a.variant == b.variant &&
                x.h == y.h && x.plasma == y.plasma && x.loss == y.loss && x.sdt == y.sdt &&
                x.inv_is == y.inv_is && x.inv_nt == y.inv_nt && x.rho_nt == y.rho_nt &&
                x.hplasma == y.hplasma && x.hloss == y.hloss && x.sat == y.sat && x.is_root == y.is_root &&
                x.K == y.K && x.nkerr == y.nkerr && x.flags == y.flags;
    for (int j = 0; j < 4; ++j) same = same && x.kerr[j] == y.kerr[j] && x.hk[j] == y.hk[j];
    return same;
}

// The launches of one block for the pulse group starting at pulse i (pulses
// i and i+1 when they share a paired column launch); *m receives the group
// size.  Groups are independent of one another.  kind -1: the group's
// column launch alone.
template <typename T>
cudaError_t launch_group(fcn_ctx *ctx, int kind, double dz, cudaStream_t st,
                         const std::vector<const cx<T> *> &tabs, const std::vector<void *> *fields,
                         size_t i, size_t *m_out, const std::vector<void *> *srcs = nullptr,
                         const std::vector<void *> *cmps = nullptr) {
    cudaError_t e = cudaSuccess;
    {
        // pulses i and i+1 share the column launch when pairing is on and
        // they have the same grid and pivot table
        const bool pair = kind != 0 && pairable(ctx, tabs, i);
        const size_t m = pair ? 2 : 1;
        *m_out = m;
        auto rows1 = [&](size_t k, int ops, int pk) {
            Pulse &pu = ctx->pulses[k];
            void *f = fields ? (*fields)[k] : pu.field;
            RowArgs<T> a = row_args<T>(pu, f, ops, dz);
            if (srcs && kind == 0) a.in = (const cx<T> *)(*srcs)[k];
            if (ops & OP_DIFF) {
                a.cmp = (const cx<T> *)(*cmps)[k];
                a.diff = pu.rows;
            }
            return timed(ctx, pk, st, [&] { return launch_rows<T>(a, pu.g.nt, st); });
        };
        // the row stage of the group's pulses (one two-pulse launch when the
        // pair's launches differ only in their buffers and mode 2 is set)
        auto rows_group = [&](int ops, int pk) {
            if (m == 2 && ctx->multi_mode == 2) {
                Pulse &p0 = ctx->pulses[i], &p1 = ctx->pulses[i + 1];
                RowMultiArgs<T> ma;
                ma.a = row_args<T>(p0, fields ? (*fields)[i] : p0.field, ops, dz);
                const RowArgs<T> a1 = row_args<T>(p1, fields ? (*fields)[i + 1] : p1.field, ops, dz);
                if (same_row_launch(ma.a, a1)) {
                    for (int c = 0; c < kRowMulti; ++c) {
                        ma.field[c] = nullptr;
                        ma.rho[c] = nullptr;
                        ma.stats[c] = nullptr;
                    }
                    ma.field[0] = ma.a.field; ma.rho[0] = ma.a.rho; ma.stats[0] = ma.a.stats;
                    ma.field[1] = a1.field; ma.rho[1] = a1.rho; ma.stats[1] = a1.stats;
                    if (ops & OP_DIFF) {
                        ma.cmp[0] = (const cx<T> *)(*cmps)[i];
                        ma.cmp[1] = (const cx<T> *)(*cmps)[i + 1];
                        ma.diff[0] = p0.rows;
                        ma.diff[1] = p1.rows;
                    }
                    return timed(ctx, pk, st, [&] { return launch_rows_multi<T>(ma, 2, p0.g.nt, st); });
                }
            }
            cudaError_t r = cudaSuccess;
            for (size_t k = i; k < i + m && r == cudaSuccess; ++k) r = rows1(k, ops, pk);
            return r;
        };
        auto col = [&] {
            Pulse &pu = ctx->pulses[i];
            void *f = fields ? (*fields)[i] : pu.field;
            if (!pair)
                return timed(ctx, FCN_PROF_COLUMN, st, [&] { return launch_cn<T>(col_args<T>(pu, f, tabs[i], dz), st); });
            void *f2 = fields ? (*fields)[i + 1] : ctx->pulses[i + 1].field;
            return timed(ctx, FCN_PROF_COLUMN, st,
                         [&] { return launch_cn_pair<T>(col_args<T>(pu, f, tabs[i], dz), (cx<T> *)f2, st); });
        };
        if (kind == -1) {
            e = col();
        } else if (kind == 0) {
            e = rows1(i, OPS_HEAD, FCN_PROF_ROW_HEAD);
        } else if (kind == 1 || kind == 2) {
            const int reps = kind == 1 ? 8 : 1;
            for (int r = 0; r < reps && e == cudaSuccess; ++r) {
                e = col();
                if (e == cudaSuccess) e = rows_group(OPS_MID, FCN_PROF_ROW_MID);
            }
        } else {
            e = col();
            const int tops = (kind == 5 ? OPS_TAIL_BARE : OPS_TAIL) | (cmps ? OP_DIFF : 0);
            if (e == cudaSuccess) e = rows_group(tops, FCN_PROF_ROW_TAIL);
        }
    }
    return e;
}

// Row stage of every pulse with operations `ops`: consecutive pulses whose
// launches differ only in their pointers go into one multi-pulse launch (at
// most kRowMulti per launch).
template <typename T>
cudaError_t launch_rows_all(fcn_ctx *ctx, int ops, int pk, double dz, cudaStream_t st,
                            const std::vector<void *> *fields, const std::vector<void *> *srcs = nullptr,
                            const std::vector<void *> *cmps = nullptr) {
    const size_t n = ctx->pulses.size();
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < n && e == cudaSuccess;) {
        Pulse &p0 = ctx->pulses[i];
        RowMultiArgs<T> m;
        m.a = row_args<T>(p0, fields ? (*fields)[i] : p0.field, ops, dz);
        int cnt = 0;
        size_t k = i;
        for (; k < n && cnt < kRowMulti; ++k) {
            Pulse &pk_ = ctx->pulses[k];
            const RowArgs<T> ak = row_args<T>(pk_, fields ? (*fields)[k] : pk_.field, ops, dz);
            if (k > i && !same_row_launch(m.a, ak)) break;
            m.field[cnt] = ak.field;
            m.rho[cnt] = ak.rho;
            m.stats[cnt] = ak.stats;
            m.in[cnt] = srcs ? (const cx<T> *)(*srcs)[k] : nullptr;
            m.cmp[cnt] = cmps ? (const cx<T> *)(*cmps)[k] : nullptr;
            m.diff[cnt] = cmps ? pk_.rows : nullptr;
            ++cnt;
        }
        m.a.in = m.in[0];
        m.a.cmp = m.cmp[0];
        m.a.diff = m.diff[0];
        for (int c = cnt; c < kRowMulti; ++c) {
            m.field[c] = nullptr;
            m.rho[c] = nullptr;
            m.stats[c] = nullptr;
            m.in[c] = nullptr;
            m.cmp[c] = nullptr;
            m.diff[c] = nullptr;
        }
        e = timed(ctx, pk, st, [&] {
            return cnt == 1 ? launch_rows<T>(m.a, p0.g.nt, st) : launch_rows_multi<T>(m, cnt, p0.g.nt, st);
        });
        i = k;
    }
    return e;
}

template <typename T>
// srcs (kind 0 only): the head reads pulse k's rows from srcs[k] and writes
// them to its field (fields[k]): out of place, no copy of the start field.
// cmps (kind 3 only): the tail also leaves the step-doubling norm's per-row
// sums of its output against cmps[k] in pulse k's rows buffer (OP_DIFF).
cudaError_t launch_block(fcn_ctx *ctx, int kind, double dz, cudaStream_t st,
                         const std::vector<const cx<T> *> &tabs,
                         const std::vector<void *> *fields = nullptr,
                         const std::vector<void *> *srcs = nullptr,
                         const std::vector<void *> *cmps = nullptr) {
    if (ctx->batched && !fields) return launch_block_batched<T>(ctx, kind, dz, st, tabs);
    if (kind != 3) cmps = nullptr;
    cudaError_t e = cudaSuccess;
    const size_t n = ctx->pulses.size();
    size_t m = 1;
    const bool seq_all = ctx->seq_all == 1 && n >= 2;
    if ((ctx->multi_mode != 1 && !seq_all) || n == 1) {
        for (size_t i = 0; i < n && e == cudaSuccess; i += m)
            e = launch_group<T>(ctx, kind, dz, st, tabs, fields, i, &m, srcs, cmps);
        return e;
    }
    // multi-pulse row launches (mode 1, and always with the sequential
    // column kernel over all pulses): per z-step the column stage of every
    // pulse group, then the row stage of all pulses (each pulse still runs
    // head, (column, row) per step and tail in order)
    if (kind == 0) return launch_rows_all<T>(ctx, OPS_HEAD, FCN_PROF_ROW_HEAD, dz, st, fields, srcs);
    const int reps = kind == 1 ? 8 : 1;
    // with the sequential column kernel chosen, all pulses (same grid and
    // pivot table) take one column launch together
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        if (seq_all) {
            std::vector<cx<T> *> f(n);
            for (size_t i = 0; i < n; ++i) f[i] = (cx<T> *)(fields ? (*fields)[i] : ctx->pulses[i].field);
            e = timed(ctx, FCN_PROF_COLUMN, st, [&] {
                return launch_cn_seq<T>(col_args<T>(ctx->pulses[0], f[0], tabs[0], dz), f.data(), (int)n, st,
                                        ctx->seq_shape);
            });
        } else {
            for (size_t i = 0; i < n && e == cudaSuccess; i += m) e = launch_group<T>(ctx, -1, dz, st, tabs, fields, i, &m);
        }
        if (e == cudaSuccess)
            e = kind == 3 || kind == 5
                    ? launch_rows_all<T>(ctx, (kind == 5 ? OPS_TAIL_BARE : OPS_TAIL) | (cmps ? OP_DIFF : 0),
                                         FCN_PROF_ROW_TAIL, dz, st, fields, nullptr, cmps)
                          : launch_rows_all<T>(ctx, OPS_MID, FCN_PROF_ROW_MID, dz, st, fields);
    }
    return e;
}

// Capture of one block with the pulse groups spread round-robin over
// ctx->branches forked streams (fork and join through events on `st`).
template <typename T>
cudaError_t launch_block_branched(fcn_ctx *ctx, int kind, double dz, cudaStream_t st,
                                  const std::vector<const cx<T> *> &tabs) {
    const int nb = ctx->branches;
    cudaError_t e = cudaEventRecord(ctx->fork_ev, st);
    for (int b = 0; b < nb && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(ctx->bst[b], ctx->fork_ev, 0);
    const size_t n = ctx->pulses.size();
    size_t m = 1;
    int g = 0;
    for (size_t i = 0; i < n && e == cudaSuccess; i += m, ++g)
        e = launch_group<T>(ctx, kind, dz, ctx->bst[g % nb], tabs, nullptr, i, &m);
    for (int b = 0; b < nb; ++b) {
        // join every branch, also after an error, so that the capture ends cleanly
        cudaError_t r = cudaEventRecord(ctx->join_ev[b], ctx->bst[b]);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(st, ctx->join_ev[b], 0);
        if (e == cudaSuccess) e = r;
    }
    return e;
}

// The timing events made during one capture: destroyed unless the graph
// is kept (release()).
struct ContextEvents {
    fcn_ctx::EvList list;
    fcn_ctx::EvList release() {
        fcn_ctx::EvList out;
        out.swap(list);
        return out;
    }
    ~ContextEvents() {
        for (auto &pe : list) {
            cudaEventDestroy(pe.second.first);
            cudaEventDestroy(pe.second.second);
        }
    }
};

template <typename T>
int run_block(fcn_ctx *ctx, int kind, double dz, const std::vector<const cx<T> *> &tabs,
              bool use_graph) {
    if (!use_graph || ctx->profiling == 1) {
        CK(launch_block<T>(ctx, kind, dz, ctx->st, tabs), "kernel launch");
        return FCN_OK;
    }
    const bool timed_graph = ctx->profiling == 2;
    GraphKey key{kind + (timed_graph ? 4 : 0), dz_key(dz)};
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        // capture on the internal stream (the legacy default stream cannot
        // be captured), then replay on the caller's stream
        cudaGraph_t g = nullptr;
        ContextEvents evs;
        CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        if (timed_graph) ctx->cap_events = &evs.list;
        cudaError_t le = (ctx->branches > 1 && !ctx->batched)
                             ? launch_block_branched<T>(ctx, kind, dz, ctx->cap, tabs)
                             : launch_block<T>(ctx, kind, dz, ctx->cap, tabs);
        ctx->cap_events = nullptr;
        cudaError_t ce = cudaStreamEndCapture(ctx->cap, &g);
        if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(ctx, le, "captured launch"); }
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "end capture");
        cudaGraphExec_t ex = nullptr;
        cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return cuda_fail(ctx, ie, "graph instantiate");
        it = ctx->graphs.emplace(key, ex).first;
        if (timed_graph) ctx->graph_events[key] = evs.release();
    }
    CK(cudaGraphLaunch(it->second, ctx->st), "graph launch");
    if (timed_graph) {
        // the graph's event nodes hold this replay's times: read them before
        // the next replay records them again
        CK(cudaStreamSynchronize(ctx->st), "timed graph sync");
        for (auto &pe : ctx->graph_events[key]) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, pe.second.first, pe.second.second), "graph event time");
            ctx->prof_ms[pe.first] += ms;
            ctx->prof_n[pe.first] += 1;
        }
    }
    return FCN_OK;
}

// ---- autotuner: kernel variants per (precision, Nr, Nt) ----
// Variants change register allocation (row stage) or the chunk length and
// CTA size (column stage); all compute the same step, the column variants
// with a different rounding order.  The first fcn_step of a grid times every
// variant on a scratch copy of the field (a few launches each, CUDA events)
// and keeps the fastest in a process-wide table, optionally persisted in the
// text file named by FCN_TUNE_CACHE ("prec nr nt row col" per line).
std::map<std::tuple<int, int, int>, std::pair<int, int>> g_tune;
bool g_tune_loaded = false;

void tune_cache_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("FCN_TUNE_CACHE");
    if (!path) return;
    std::ifstream f(path);
    int prec, nr, nt, rv, cv;
    while (f >> prec >> nr >> nt >> rv >> cv)
        if (rv >= 0 && rv < kRowVariants && cv >= 0 && cv < kColVariants)
            g_tune[std::make_tuple(prec, nr, nt)] = {rv, cv};
}

void tune_cache_store(int prec, int nr, int nt, int rv, int cv) {
    const char *path = std::getenv("FCN_TUNE_CACHE");
    if (!path) return;
    std::ofstream f(path, std::ios::app);
    f << prec << " " << nr << " " << nt << " " << rv << " " << cv << "\n";
}

// 3 untimed then 15 timed launches (variants differ by a few per cent, so
// a shorter sample lets launch-to-launch noise decide)
template <typename F>
int time_launches(fcn_ctx *ctx, F &&launch, float *ms_out) {
    for (int i = 0; i < 3; ++i) CK(launch(), "tuning warm-up");
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    cudaEventRecord(e0, ctx->st);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 15 && e == cudaSuccess; ++i) e = launch();
    cudaEventRecord(e1, ctx->st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tuning launch");
    *ms_out = ms;
    return FCN_OK;
}

template <typename T>
int tune_pulse(fcn_ctx *ctx, Pulse &pu, const cx<T> *tab, double dz) {
    const int prec = ctx->prec;
    std::lock_guard<std::mutex> lk(g_mu);
    tune_cache_load();
    auto key = std::make_tuple(prec, pu.g.nr, pu.g.nt);
    auto it = g_tune.find(key);
    if (it == g_tune.end()) {
        // a private scratch copy: the context's work buffers may hold state
        const size_t bytes = csize(prec) * pu.points();
        void *scratch = nullptr;
        CK(cudaMalloc(&scratch, bytes), "tuning scratch");
        struct Free {
            void *p;
            ~Free() { cudaFree(p); }
        } guard{scratch};
        CK(cudaMemcpyAsync(scratch, pu.field, bytes, cudaMemcpyDeviceToDevice, ctx->st), "tuning copy");
        // three interleaved rounds over the variants, each variant's best
        // round counts (a burst of noise on the GPU then decides nothing)
        const int nrv = (sizeof(T) == 4 && pu.p.K == 8) ? kRowVariants : 1;
        std::vector<float> tr(nrv, 1e30f), tc(kColVariants, 1e30f);
        for (int round = 0; round < 3; ++round) {
            for (int v = 0; v < nrv; ++v) {
                RowArgs<T> a = row_args<T>(pu, scratch, OPS_MID, dz);
                a.variant = v;
                float ms;
                int rc = time_launches(ctx, [&] { return launch_rows<T>(a, pu.g.nt, ctx->st); }, &ms);
                if (rc) return rc;
                tr[v] = std::min(tr[v], ms);
            }
            for (int v = 0; v < kColVariants; ++v) {
                ColArgs<T> a = col_args<T>(pu, scratch, tab, dz);
                a.variant = v;
                float ms;
                int rc = time_launches(ctx, [&] { return launch_cn<T>(a, ctx->st); }, &ms);
                if (rc) return rc;
                tc[v] = std::min(tc[v], ms);
            }
        }
        const int best_r = int(std::min_element(tr.begin(), tr.end()) - tr.begin());
        const int best_c = int(std::min_element(tc.begin(), tc.end()) - tc.begin());
        CK(cudaStreamSynchronize(ctx->st), "tuning sync");
        it = g_tune.emplace(key, std::make_pair(best_r, best_c)).first;
        tune_cache_store(prec, pu.g.nr, pu.g.nt, best_r, best_c);
    }
    pu.row_var = ctx->force_row >= 0 ? ctx->force_row : it->second.first;
    pu.col_var = ctx->force_col >= 0 ? ctx->force_col : it->second.second;
    pu.tuned = true;
    return FCN_OK;
}

template <typename T>
int ensure_tuned(fcn_ctx *ctx, const std::vector<const cx<T> *> &tabs, double dz) {
    if (ctx->batched) return FCN_OK;   // the work-list kernels have a single variant
    for (size_t i = 0; i < ctx->pulses.size(); ++i) {
        Pulse &pu = ctx->pulses[i];
        if (pu.tuned) continue;
        if (ctx->force_row >= 0 && ctx->force_col >= 0) {
            pu.row_var = ctx->force_row;
            pu.col_var = ctx->force_col;
            pu.tuned = true;
            continue;
        }
        int rc = tune_pulse<T>(ctx, pu, tabs[i], dz);
        if (rc) return rc;
    }
    if (ctx->pairs < 0) {
        ctx->pairs = 0;
        bool eligible = sizeof(T) == 4 && ctx->pulses.size() >= 2;
        for (size_t i = 1; eligible && i < ctx->pulses.size(); ++i)
            eligible = ctx->pulses[i].g.nr == ctx->pulses[0].g.nr && ctx->pulses[i].g.nt == ctx->pulses[0].g.nt &&
                       tabs[i] == tabs[0];
        if (eligible && ctx->pair_mode == 1) ctx->pairs = 1;
        if (eligible && ctx->pair_mode == -1) {
            // one paired launch against the tuned single launch twice, on
            // private scratch copies of the first pulse
            Pulse &pu = ctx->pulses[0];
            const size_t bytes = csize(ctx->prec) * pu.points();
            void *s1 = nullptr, *s2 = nullptr;
            CK(cudaMalloc(&s1, bytes), "pairing scratch");
            struct Free {
                void *p;
                ~Free() { cudaFree(p); }
            } g1{s1};
            CK(cudaMalloc(&s2, bytes), "pairing scratch");
            Free g2{s2};
            CK(cudaMemcpyAsync(s1, pu.field, bytes, cudaMemcpyDeviceToDevice, ctx->st), "pairing copy");
            CK(cudaMemcpyAsync(s2, pu.field, bytes, cudaMemcpyDeviceToDevice, ctx->st), "pairing copy");
            float t_pair = 0.f, t_single = 0.f;
            int rc = time_launches(ctx, [&] {
                return launch_cn_pair<T>(col_args<T>(pu, s1, tabs[0], dz), (cx<T> *)s2, ctx->st);
            }, &t_pair);
            if (rc) return rc;
            rc = time_launches(ctx, [&] {
                cudaError_t e = launch_cn<T>(col_args<T>(pu, s1, tabs[0], dz), ctx->st);
                return e == cudaSuccess ? launch_cn<T>(col_args<T>(pu, s2, tabs[0], dz), ctx->st) : e;
            }, &t_single);
            if (rc) return rc;
            CK(cudaStreamSynchronize(ctx->st), "pairing sync");
            ctx->pairs = t_pair < t_single ? 1 : 0;
        }
    }
    if (ctx->seq_all < 0) {
        ctx->seq_all = 0;
        const size_t n = ctx->pulses.size();
        Pulse &p0 = ctx->pulses[0];
        bool eligible = n >= 2 && n <= 8 && ctx->branches == 1 && ctx->seq_mode != 0 &&
                        cn_seq_supported<T>(col_args<T>(p0, p0.field, tabs[0], dz));
        for (size_t i = 1; eligible && i < n; ++i)
            eligible = ctx->pulses[i].g.nr == p0.g.nr && ctx->pulses[i].g.nt == p0.g.nt && tabs[i] == tabs[0];
        if (eligible && ctx->seq_mode == 1) ctx->seq_all = 1;
        if (eligible && ctx->seq_mode == -1) {
            // one launch over all pulses against the per-group launches of
            // the tuned variants, on private scratch copies of the fields
            const size_t bytes = csize(ctx->prec) * p0.points();
            void *scratch = nullptr;
            CK(cudaMalloc(&scratch, bytes * n), "sequential-column scratch");
            struct Free {
                void *p;
                ~Free() { cudaFree(p); }
            } guard{scratch};
            std::vector<void *> f(n);
            std::vector<cx<T> *> fc(n);
            for (size_t i = 0; i < n; ++i) {
                f[i] = (char *)scratch + i * bytes;
                fc[i] = (cx<T> *)f[i];
                CK(cudaMemcpyAsync(f[i], ctx->pulses[i].field, bytes, cudaMemcpyDeviceToDevice, ctx->st),
                   "sequential-column copy");
            }
            float t_all = 1e30f, t_groups = 0.f;
            int rc = 0;
            for (int shape = 0; shape < kSeqShapes; ++shape) {
                float t = 0.f;
                rc = time_launches(ctx, [&] {
                    return launch_cn_seq<T>(col_args<T>(p0, f[0], tabs[0], dz), fc.data(), (int)n, ctx->st, shape);
                }, &t);
                if (rc) return rc;
                if (t < t_all) {
                    t_all = t;
                    ctx->seq_shape = shape;
                }
            }
            rc = time_launches(ctx, [&] {
                cudaError_t e = cudaSuccess;
                size_t m = 1;
                for (size_t i = 0; i < n && e == cudaSuccess; i += m) e = launch_group<T>(ctx, -1, dz, ctx->st, tabs, &f, i, &m);
                return e;
            }, &t_groups);
            if (rc) return rc;
            CK(cudaStreamSynchronize(ctx->st), "sequential-column sync");
            ctx->seq_all = t_all < t_groups ? 1 : 0;
        }
    }
    return FCN_OK;
}

template <typename T>
int step_impl(fcn_ctx *ctx, double dz, int64_t n, bool use_graph) {
    if (!(dz > 0) || !std::isfinite(dz)) return fail(ctx, FCN_ERR_ARG, "dz must be > 0 and finite");
    if (n < 0) return fail(ctx, FCN_ERR_ARG, "n must be >= 0");
    for (auto &pu : ctx->pulses)
        if (!pu.has_field) return fail(ctx, FCN_ERR_STATE, "fcn_set_field has not been called");
    if (n == 0) return FCN_OK;
    std::vector<const cx<T> *> tabs(ctx->pulses.size());
    for (size_t i = 0; i < ctx->pulses.size(); ++i) {
        int rc = ensure_table<T>(ctx, ctx->pulses[i], dz, &tabs[i]);
        if (rc) return rc;
    }
    {
        int rc = ensure_tuned<T>(ctx, tabs, dz);
        if (rc) return rc;
    }
    if (ctx->batched) {
        // argument arrays are copied synchronously: never inside a capture
        const RowArgs<T> *ra;
        const ColArgs<T> *ca;
        CK(batch_args<T>(ctx, dz, tabs, &ra, &ca), "batch arguments");
    }
    int rc = run_block<T>(ctx, 0, dz, tabs, use_graph);
    int64_t rem = n - 1;
    while (rc == FCN_OK && rem >= 8) { rc = run_block<T>(ctx, 1, dz, tabs, use_graph); rem -= 8; }
    while (rc == FCN_OK && rem >= 1) { rc = run_block<T>(ctx, 2, dz, tabs, use_graph); rem -= 1; }
    if (rc == FCN_OK) rc = run_block<T>(ctx, 3, dz, tabs, use_graph);
    if (rc) return rc;
    for (auto &pu : ctx->pulses) {
        pu.z += dz * double(n);
        pu.steps += n;
    }
    return FCN_OK;
}

// One Strang step of length h (or two of h/2) on a work buffer, direct launches.
template <typename T>
int substeps(fcn_ctx *ctx, Pulse &pu, void *f, double h, int count, const cx<T> *tab = nullptr,
             cudaEvent_t table_ready = nullptr, int tail_ops = OPS_TAIL, const void *src = nullptr,
             const void *cmp = nullptr) {
    if (!tab) {
        int rc = ensure_table<T>(ctx, pu, h, &tab);
        if (rc) return rc;
    }
    if (!pu.tuned) {
        std::vector<const cx<T> *> tabs(ctx->pulses.size(), tab);
        int rc = ensure_tuned<T>(ctx, tabs, h);
        if (rc) return rc;
    }
    {
        // src: the head reads its rows there and writes them to f (out of
        // place: the field an attempt starts from needs no copy)
        RowArgs<T> a = row_args<T>(pu, f, OPS_HEAD, h);
        a.in = (const cx<T> *)src;
        CK(launch_rows<T>(a, pu.g.nt, ctx->st), "head");
    }
    // the opening row stage does not read the table: a table built on a side
    // stream has until here
    if (table_ready) CK(cudaStreamWaitEvent(ctx->st, table_ready, 0), "table wait");
    for (int i = 0; i < count; ++i) {
        CK(launch_cn<T>(col_args<T>(pu, f, tab, h), ctx->st), "column");
        const int ops = (i + 1 < count) ? OPS_MID : tail_ops;
        RowArgs<T> a = row_args<T>(pu, f, ops, h);
        if (cmp && i + 1 == count) {
            // the closing launch also leaves the per-row norm sums against cmp
            a.ops |= OP_DIFF;
            a.cmp = (const cx<T> *)cmp;
            a.diff = pu.rows;
        }
        CK(launch_rows<T>(a, pu.g.nt, ctx->st), "row");
    }
    return FCN_OK;
}

template <typename T>
int diag_impl(fcn_ctx *ctx, Pulse &pu, fcn_diag *out) {
    RowArgs<T> a = row_args<T>(pu, pu.field, OP_STATS | OP_FFT | OP_SPEC | OP_NOSTORE, 0.0);
    a.variant = 0;
    CK(launch_rows<T>(a, pu.g.nt, ctx->st), "diagnostics row pass");
    CK(launch_reduce_stats(pu.stats, pu.g.nr, pu.red, ctx->st), "diagnostics reduction");
    CK(cudaMemcpyAsync(ctx->host_red, pu.red, sizeof(double) * 8, cudaMemcpyDeviceToHost, ctx->st),
       "diagnostics copy");
    CK(cudaStreamSynchronize(ctx->st), "diagnostics sync");
    const double *r = ctx->host_red;
    const Consts c = derive(pu.g, pu.p);
    std::memset(out, 0, sizeof(*out));
    out->z = pu.z;
    out->energy = 2.0 * kPi * c.dr * c.dr * c.dtau * r[0];
    out->peak_intensity = r[1];
    out->peak_rho = r[2] * pu.p.rho_nt;
    out->onaxis_peak = r[3];
    if (r[4] > 0) {
        const double mean = r[5] / r[4];
        const double var = r[6] / r[4] - mean * mean;
        out->spectral_rms = var > 0 ? std::sqrt(var) * c.domega : 0.0;
    }
    out->steps = pu.steps;
    out->rejected = pu.rejected;
    out->nonfinite = (r[7] > 0 || !std::isfinite(r[0])) ? 1 : 0;
    return out->nonfinite ? fail(ctx, FCN_ERR_NONFINITE, "field holds NaN or Inf") : FCN_OK;
}

// Runs the diagnostic row pass and the reduction on the field; the result
// stays on the device in pu.red (see launch_reduce_stats).
template <typename T>
int diag_device(fcn_ctx *ctx, Pulse &pu, void *field) {
    RowArgs<T> a = row_args<T>(pu, field, OP_STATS | OP_FFT | OP_SPEC | OP_NOSTORE, 0.0);
    a.variant = 0;
    CK(launch_rows<T>(a, pu.g.nt, ctx->st), "diagnostics row pass");
    CK(launch_reduce_stats(pu.stats, pu.g.nr, pu.red, ctx->st), "diagnostics reduction");
    return FCN_OK;
}

// After an MLP proposal is rejected, the next kMlpCooldown accepted steps
// take the step-doubling law's proposal: a state where the network
// overreaches does not turn into a run of rejected attempts.
constexpr int kMlpCooldown = 16;

// Step doubling (controller 0) or MLP proposals judged by step doubling
// (controller 1).  With a log buffer (fcn_mlp_set_log) every attempt appends
// [f0..f5, log(h/L_ref), log(err/rtol)] for training.
// Adaptive propagation of every pulse of a multi-pulse context with one
// common dz: each attempt runs one step of h and two of h/2 on all pulses
// (the launch structure of fcn_step: one launch per stage for pulses that
// share it), and is accepted when every pulse's step-doubling error is
// within rtol, so the batch moves at the pace of its hardest pulse.  The
// law's proposal follows the largest error; the learned controller
// proposes, per pulse, from that pulse's features, and the smallest
// proposal is taken.  Counters: an accepted attempt is one accepted step of
// every pulse.
template <typename T>
int propagate_batch(fcn_ctx *ctx, double z_end, double dz0, double rtol, double dz_min, int max_reject,
                    int controller, fcn_stats *out) {
    const size_t n = ctx->pulses.size();
    for (auto &pu : ctx->pulses)
        if (!pu.has_field) return fail(ctx, FCN_ERR_STATE, "fcn_set_field has not been called");
    if (!(dz0 > 0) || !std::isfinite(dz0) || !(rtol > 0) || !std::isfinite(z_end) || !(dz_min > 0))
        return fail(ctx, FCN_ERR_ARG, "bad adaptive arguments");
    if (controller != 0 && controller != 1) return fail(ctx, FCN_ERR_ARG, "controller must be 0 or 1");
    if (controller == 1 && !ctx->has_mlp) return fail(ctx, FCN_ERR_STATE, "controller 1 needs MLP weights");
    if (ctx->batched) return fail(ctx, FCN_ERR_UNSUPPORTED, "adaptive batches use per-pulse launches (batching 0)");
    for (auto &pu : ctx->pulses)
        if (pu.z != ctx->pulses[0].z) return fail(ctx, FCN_ERR_STATE, "the pulses of a batch must be at one z");
    {
        std::vector<const cx<T> *> tabs(n);
        for (size_t i = 0; i < n; ++i) {
            int rc = ensure_table<T>(ctx, ctx->pulses[i], dz0, &tabs[i]);
            if (rc) return rc;
        }
        int rc = ensure_tuned<T>(ctx, tabs, dz0);
        if (rc) return rc;
    }
    bool same_grid = true;
    for (auto &pu : ctx->pulses)
        same_grid = same_grid && pu.g.nr == ctx->pulses[0].g.nr && pu.g.nt == ctx->pulses[0].g.nt &&
                    pu.g.r_max == ctx->pulses[0].g.r_max && pu.g.t_window == ctx->pulses[0].g.t_window &&
                    pu.p.n0 == ctx->pulses[0].p.n0 && pu.p.lambda0 == ctx->pulses[0].p.lambda0 &&
                    pu.p.k2 == ctx->pulses[0].p.k2 && pu.p.flags == ctx->pulses[0].p.flags;
    for (auto &pu : ctx->pulses) {
        const size_t bytes = csize(ctx->prec) * pu.points();
        if (!pu.work1) CK(cudaMalloc(&pu.work1, bytes), "work buffer");
        if (!pu.work2) CK(cudaMalloc(&pu.work2, bytes), "work buffer");
    }
    const bool features = controller == 1;
    // per pulse: the controller kernel's output (8 doubles) on the device and
    // its copy on the host (norms, features, proposal, energy).  Regrown
    // when pulses were added since the last batch.
    if (ctx->batch_cap < n) {
        cudaFree(ctx->batch_io);
        if (ctx->host_ctl) cudaFreeHost(ctx->host_ctl);
        ctx->batch_io = nullptr;
        ctx->host_ctl = nullptr;
        ctx->batch_cap = 0;
        CK(cudaMalloc(&ctx->batch_io, 64 * n), "controller buffer");
        CK(cudaMallocHost(&ctx->host_ctl, 16 * sizeof(double) * n), "controller buffer");
        ctx->batch_cap = n;
    }
    double *H = ctx->host_ctl;
    std::vector<MlpScalars> sc(n);
    std::vector<float> peak(n, 0.f);
    for (size_t i = 0; i < n; ++i) {
        Pulse &pu = ctx->pulses[i];
        const Consts cs = derive(pu.g, pu.p);
        std::memset(&sc[i], 0, sizeof(MlpScalars));
        sc[i].rtol = rtol;
        sc[i].l_ref = cs.k0 * (pu.g.r_max / 5.0) * (pu.g.r_max / 5.0) / 2.0;
        sc[i].domega = cs.domega;
    }
    if (features) {
        for (size_t i = 0; i < n; ++i) {
            Pulse &pu = ctx->pulses[i];
            int rc = diag_device<T>(ctx, pu, pu.field);
            if (rc) return rc;
            CK(cudaMemcpyAsync(H + 8 * i, pu.red, 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st), "ref copy");
        }
        CK(cudaStreamSynchronize(ctx->st), "ref sync");
        for (size_t i = 0; i < n; ++i) {
            sc[i].i_ref = H[8 * i + 1] > 0 ? H[8 * i + 1] : 1.0;
            sc[i].peak_prev = sc[i].i_ref;
            peak[i] = (float)sc[i].i_ref;
            sc[i].e_prev = H[8 * i];
            sc[i].dz_prev = dz0;
            sc[i].err_prev = rtol;
        }
    }
    fcn_stats s;
    std::memset(&s, 0, sizeof s);
    double z = ctx->pulses[0].z, dz = dz0;
    int consecutive = 0, cooldown = 0, status = FCN_OK;
    bool from_mlp = false;
    std::vector<void *> f0(n), f1(n), f2(n);
    std::vector<const cx<T> *> tab1(n), tab2(n);
    while (z < z_end) {
        double h = dz;
        bool last = false;
        if (z + h >= z_end) { h = z_end - z; last = true; }
        // pivot tables of h and h/2: for a batch on one grid, on side streams
        // behind the copies and the opening row stages
        cudaEvent_t ev1 = nullptr, ev2 = nullptr;
        for (size_t i = 0; i < n; ++i) {
            Pulse &pu = ctx->pulses[i];
            const int side1 = same_grid && i == 0 ? 0 : -1, side2 = same_grid && i == 0 ? 1 : -1;
            int rc = ensure_table<T>(ctx, pu, h, &tab1[i], side1, side1 >= 0 ? &ev1 : nullptr);
            if (!rc) rc = ensure_table<T>(ctx, pu, 0.5 * h, &tab2[i], side2, side2 >= 0 ? &ev2 : nullptr);
            if (rc) return rc;
            f1[i] = pu.work1;
            f2[i] = pu.work2;
            f0[i] = pu.field;
        }
        // the heads read the start field and write the work buffers
        CK(launch_block<T>(ctx, 0, h, ctx->st, tab1, &f1, &f0), "head");
        if (ev1) CK(cudaStreamWaitEvent(ctx->st, ev1, 0), "table wait");
        CK(launch_block<T>(ctx, 5, h, ctx->st, tab1, &f1), "one step");
        CK(launch_block<T>(ctx, 0, 0.5 * h, ctx->st, tab2, &f2, &f0), "head");
        if (ev2) CK(cudaStreamWaitEvent(ctx->st, ev2, 0), "table wait");
        CK(launch_block<T>(ctx, 2, 0.5 * h, ctx->st, tab2, &f2), "first half step");
        // the closing launch also leaves each pulse's per-row norm sums of
        // work2 against work1 (OP_DIFF): no pass of its own over both fields
        CK(launch_block<T>(ctx, 3, 0.5 * h, ctx->st, tab2, &f2, nullptr, &f1), "second half step");
        const bool next_feat = features && !last;
        if (same_grid && n <= (size_t)kCtlMulti) {
            // every pulse's norm, features and (no cooldown) proposals in one
            // launch, one copy
            CtlMulti cm;
            std::memset(&cm, 0, sizeof cm);
            cm.nr = ctx->pulses[0].g.nr;
            cm.n = (int)n;
            cm.out = reinterpret_cast<double *>(ctx->batch_io);
            for (size_t i = 0; i < n; ++i) {
                Pulse &pu = ctx->pulses[i];
                cm.stats[i] = pu.stats;
                cm.rows[i] = pu.rows;
                if (next_feat) {
                    sc[i].peak_prev = peak[i];
                    sc[i].dz_prev = h;
                    sc[i].dz_lo = std::fmax(0.2 * h, dz_min);
                    sc[i].dz_hi = 2.0 * h;
                }
                cm.sc[i] = sc[i];
            }
            CK(launch_mlp_step_control_multi(cm, next_feat && cooldown == 0 ? ctx->mlp : nullptr, ctx->st),
               "controller");
            CK(cudaMemcpyAsync(H, ctx->batch_io, 8 * sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->st),
               "controller copy");
        }
        for (size_t i = 0; i < n && !(same_grid && n <= (size_t)kCtlMulti); ++i) {
            Pulse &pu = ctx->pulses[i];
            if (next_feat) {
                // the closing row launch left this pulse's statistics of work2
                // and its per-row norm sums: norm, features, proposal and
                // energy in one kernel and one copy; the network runs only
                // when its proposal can be taken (no cooldown)
                sc[i].peak_prev = peak[i];
                sc[i].dz_prev = h;
                sc[i].dz_lo = std::fmax(0.2 * h, dz_min);
                sc[i].dz_hi = 2.0 * h;
                double *ctl = reinterpret_cast<double *>(ctx->batch_io + 64 * i);
                CK(launch_mlp_step_control(pu.stats, pu.g.nr, pu.rows, sc[i], cooldown == 0 ? ctx->mlp : nullptr,
                                           ctl, ctx->st),
                   "controller");
                CK(cudaMemcpyAsync(H + 8 * i, ctl, 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st),
                   "controller copy");
            } else {
                CK(launch_diff_final(pu.rows, pu.g.nr, pu.red, ctx->st), "error norm");
                CK(cudaMemcpyAsync(H + 8 * i, pu.red, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st),
                   "norm copy");
            }
        }
        CK(cudaStreamSynchronize(ctx->st), "norm sync");
        double err = 0.0;
        std::vector<double> erri(n);
        for (size_t i = 0; i < n; ++i) {
            erri[i] = H[8 * i + 1] > 0 ? std::sqrt(H[8 * i] / H[8 * i + 1]) : std::sqrt(H[8 * i]);
            if (!std::isfinite(erri[i])) err = erri[i];
            else if (std::isfinite(err)) err = std::fmax(err, erri[i]);
        }
        s.substeps += 3;
        s.last_err = err;
        if (!std::isfinite(err)) { status = fail(ctx, FCN_ERR_NONFINITE, "non-finite step-doubling error"); break; }
        double fac = err > 0 ? 0.9 * std::cbrt(rtol / err) : 2.0;
        fac = fac < 0.2 ? 0.2 : (fac > 2.0 ? 2.0 : fac);
        if (err <= rtol) {
            z = last ? z_end : z + h;
            for (size_t i = 0; i < n; ++i) {
                Pulse &pu = ctx->pulses[i];
                std::swap(pu.field, pu.work2);
                pu.z = z;
                pu.steps++;
            }
            s.accepted++;
            if (from_mlp) s.mlp_proposals++;
            consecutive = 0;
            dz = last ? dz : h * fac;
            bool proposed = false;
            if (next_feat) {
                double prop = 0.0;
                for (size_t i = 0; i < n; ++i) {
                    float hf[8];
                    std::memcpy(hf, H + 8 * i + 2, sizeof hf);
                    peak[i] = hf[7];
                    sc[i].err_prev = erri[i];
                    sc[i].e_prev = H[8 * i + 7];
                    const double p = H[8 * i + 6];
                    if (std::isfinite(p) && p > 0) prop = prop > 0 ? std::fmin(prop, p) : p;
                }
                if (cooldown > 0) {
                    --cooldown;
                } else if (prop > 0) {
                    dz = prop;
                    proposed = true;
                }
            }
            from_mlp = proposed && z < z_end;
        } else {
            for (auto &pu : ctx->pulses) pu.rejected++;
            s.rejected++;
            consecutive++;
            dz = h * fac;          // the step-doubling formula is the fallback
            if (from_mlp) cooldown = kMlpCooldown;
            from_mlp = false;
        }
        if (dz < dz_min || consecutive > max_reject) {
            status = fail(ctx, FCN_ERR_STEP_UNDERFLOW, "dz underflow or too many rejections");
            break;
        }
    }
    for (auto &pu : ctx->pulses) pu.dz_next = dz;
    s.z = z;
    s.dz_next = dz;
    if (out) *out = s;
    return status;
}

template <typename T>
int propagate_impl(fcn_ctx *ctx, double z_end, double dz0, double rtol, double dz_min,
                   int max_reject, int controller, fcn_stats *out) {
    if (ctx->pulses.size() != 1) return propagate_batch<T>(ctx, z_end, dz0, rtol, dz_min, max_reject, controller, out);
    Pulse &pu = ctx->pulses[0];
    if (!pu.has_field) return fail(ctx, FCN_ERR_STATE, "fcn_set_field has not been called");
    if (!(dz0 > 0) || !std::isfinite(dz0) || !(rtol > 0) || !std::isfinite(z_end) || !(dz_min > 0))
        return fail(ctx, FCN_ERR_ARG, "bad adaptive arguments");
    if (controller != 0 && controller != 1) return fail(ctx, FCN_ERR_ARG, "controller must be 0 or 1");
    if (controller == 1 && !ctx->has_mlp) return fail(ctx, FCN_ERR_STATE, "controller 1 needs MLP weights");
    const size_t bytes = csize(ctx->prec) * pu.points();
    if (!pu.tuned) {
        const cx<T> *tab = nullptr;
        int rc = ensure_table<T>(ctx, pu, dz0, &tab);
        if (rc) return rc;
        std::vector<const cx<T> *> tabs(1, tab);
        rc = ensure_tuned<T>(ctx, tabs, dz0);
        if (rc) return rc;
    }
    if (!pu.work1) CK(cudaMalloc(&pu.work1, bytes), "work buffer");
    if (!pu.work2) CK(cudaMalloc(&pu.work2, bytes), "work buffer");
    const bool features = controller == 1 || ctx->log_buf != nullptr;
    if (features && !ctx->mlp_io) CK(cudaMalloc(&ctx->mlp_io, 64), "controller buffer");
    const Consts cs = derive(pu.g, pu.p);
    MlpScalars sc;
    std::memset(&sc, 0, sizeof sc);
    sc.rtol = rtol;
    sc.l_ref = cs.k0 * (pu.g.r_max / 5.0) * (pu.g.r_max / 5.0) / 2.0;
    sc.domega = cs.domega;
    // hfeat: f0..f5, fE and the peak intensity of the current state.  The
    // controller kernel leaves [norm0, norm1, hfeat (4 doubles), proposal,
    // energy sum] in ctl_d, which comes back in one copy into host_red[0..7]
    float hfeat[8] = {0};
    double mlp_dz = 0.0;
    double *ctl_d = reinterpret_cast<double *>(ctx->mlp_io);
    if (features) {
        // references from the field at the start of the run
        int rc = diag_device<T>(ctx, pu, pu.field);
        if (rc) return rc;
        CK(cudaMemcpyAsync(ctx->host_red, pu.red, 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st), "ref copy");
        CK(cudaStreamSynchronize(ctx->st), "ref sync");
        sc.i_ref = ctx->host_red[1] > 0 ? ctx->host_red[1] : 1.0;
        sc.peak_prev = sc.i_ref;
        sc.e_prev = ctx->host_red[0];
        sc.dz_prev = dz0;
        sc.err_prev = rtol;
        CK(launch_mlp_step_control(pu.stats, pu.g.nr, nullptr, sc, nullptr, ctl_d, ctx->st), "features");
        CK(cudaMemcpyAsync(ctx->host_red, ctl_d, 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st),
           "features copy");
        CK(cudaStreamSynchronize(ctx->st), "features sync");
        std::memcpy(hfeat, ctx->host_red + 2, 8 * sizeof(float));
    }
    fcn_stats s;
    std::memset(&s, 0, sizeof s);
    double dz = dz0;
    int consecutive = 0, cooldown = 0;
    int status = FCN_OK;
    bool from_mlp = false;
    while (pu.z < z_end) {
        double h = dz;
        bool last = false;
        if (pu.z + h >= z_end) { h = z_end - pu.z; last = true; }
        // the pivot tables of h and h/2 (new at almost every attempt) build on
        // side streams, side by side and behind the copies and opening row
        // stages; the column stages wait for them
        const cx<T> *tab1 = nullptr, *tab2 = nullptr;
        cudaEvent_t ev1 = nullptr, ev2 = nullptr;
        int rc = ensure_table<T>(ctx, pu, h, &tab1, 0, &ev1);
        if (!rc) rc = ensure_table<T>(ctx, pu, 0.5 * h, &tab2, 1, &ev2);
        if (rc) return rc;
        // the heads read the start field and write the work buffers (no copies)
        // (the one-step result only enters the error norm: a bare tail)
        rc = substeps<T>(ctx, pu, pu.work1, h, 1, tab1, ev1, OPS_TAIL_BARE, pu.field);
        // the closing launch of the two half steps leaves the statistics of
        // the field it produces (peak, on-axis peak, peak rho, energy), from
        // which the features and the proposal of an accepted attempt follow
        // without a pass of their own
        const bool next_feat = features && !last;
        if (!rc) rc = substeps<T>(ctx, pu, pu.work2, 0.5 * h, 2, tab2, ev2, OPS_TAIL, pu.field, pu.work1);
        if (rc) return rc;
        if (next_feat) {
            // the norm, the features of work2 and (speculative, used only
            // if the attempt is accepted) the proposal after it: one kernel
            // over the per-row norm sums the closing launch left, one copy.
            // The network runs only when its proposal can be taken (no
            // cooldown).
            sc.peak_prev = hfeat[7];
            sc.dz_prev = h;
            sc.dz_lo = std::fmax(0.2 * h, dz_min);
            sc.dz_hi = 2.0 * h;
            CK(launch_mlp_step_control(pu.stats, pu.g.nr, pu.rows, sc,
                                       controller == 1 && cooldown == 0 ? ctx->mlp : nullptr, ctl_d, ctx->st),
               "controller");
            CK(cudaMemcpyAsync(ctx->host_red, ctl_d, 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st),
               "controller copy");
        } else {
            CK(launch_diff_final(pu.rows, pu.g.nr, pu.red, ctx->st), "error norm");
            CK(cudaMemcpyAsync(ctx->host_red, pu.red, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st),
               "norm copy");
        }
        CK(cudaStreamSynchronize(ctx->st), "norm sync");
        const double err = ctx->host_red[1] > 0 ? std::sqrt(ctx->host_red[0] / ctx->host_red[1])
                                                : std::sqrt(ctx->host_red[0]);
        s.substeps += 3;
        s.last_err = err;
        if (!std::isfinite(err)) { status = fail(ctx, FCN_ERR_NONFINITE, "non-finite step-doubling error"); break; }
        if (ctx->log_buf && ctx->log_n < ctx->log_cap) {
            float *rec = ctx->log_buf + FCN_MLP_LOG_FLOATS * ctx->log_n;
            for (int k = 0; k < 7; ++k) rec[k] = hfeat[k];
            rec[7] = (float)std::log(h / sc.l_ref);
            rec[8] = (float)std::log(std::fmax(err, 1e-30) / rtol);
            ctx->log_n++;
        }
        double fac = err > 0 ? 0.9 * std::cbrt(rtol / err) : 2.0;
        fac = fac < 0.2 ? 0.2 : (fac > 2.0 ? 2.0 : fac);
        const bool accepted = err <= rtol;
        if (accepted) {
            std::swap(pu.field, pu.work2);
            pu.z = last ? z_end : pu.z + h;
            pu.steps++;
            s.accepted++;
            if (from_mlp) s.mlp_proposals++;
            consecutive = 0;
            dz = last ? dz : h * fac;
            bool proposed = false;
            if (next_feat) {
                std::memcpy(hfeat, ctx->host_red + 2, 8 * sizeof(float));
                sc.err_prev = err;
                sc.e_prev = ctx->host_red[7];
                if (controller == 1) {
                    mlp_dz = ctx->host_red[6];
                    if (cooldown > 0) {
                        --cooldown;
                    } else if (std::isfinite(mlp_dz) && mlp_dz > 0) {
                        dz = mlp_dz;
                        proposed = true;
                    }
                }
            }
            from_mlp = proposed && pu.z < z_end;
        } else {
            pu.rejected++;
            s.rejected++;
            consecutive++;
            dz = h * fac;          // the step-doubling formula is the fallback
            if (from_mlp) cooldown = kMlpCooldown;
            from_mlp = false;
        }
        if (dz < dz_min || consecutive > max_reject) {
            status = fail(ctx, FCN_ERR_STEP_UNDERFLOW, "dz underflow or too many rejections");
            break;
        }
    }
    pu.dz_next = dz;
    s.z = pu.z;
    s.dz_next = dz;
    if (out) *out = s;
    return status;
}

Pulse *get_pulse(fcn_ctx *ctx, int pulse) {
    if (!ctx || pulse < 0 || pulse >= (int)ctx->pulses.size()) return nullptr;
    return &ctx->pulses[pulse];
}

// Work lists of the batched kernels: row items (pulse, first row) with
// 512/(Nt/16) rows each, column items (pulse, group, C) with C P <= 512 (P =
// chunks of 16 rows); both sorted largest first.  Only when every pulse runs
// FP32 with K = 8 and Nt >= 512 (else per-pulse launches are used).
int setup_batch(fcn_ctx *ctx) {
    for (auto &pu : ctx->pulses)
        if (pu.p.K != 8 || pu.g.nt < 512) return FCN_OK;
    if (ctx->row_items) return FCN_OK;   // already built
    std::vector<std::pair<int64_t, int2>> rows;
    std::vector<std::pair<int64_t, int4>> cols;
    size_t smem = 0;
    for (size_t i = 0; i < ctx->pulses.size(); ++i) {
        const Pulse &pu = ctx->pulses[i];
        const int nt = pu.g.nt, nr = pu.g.nr;
        const int rpi = 512 / (nt / 16);
        for (int r0 = 0; r0 < nr; r0 += rpi) rows.push_back({(int64_t)nt, make_int2((int)i, r0)});
        const size_t sm = row_batch_smem(nt, 8);
        if (sm > smem) smem = sm;
        const int P = (nr + 15) / 16;
        int C = 4;
        while (C * 2 * P <= 512 && C * 2 <= 32) C *= 2;
        if (C > nt) C = nt;
        const int ng = nt / C;
        for (int b = 0; b < ng; ++b) {
            const int g = (b & 1) ? (ng - 1 - (b >> 1)) : (b >> 1);
            cols.push_back({(int64_t)nr * C, make_int4((int)i, g, C, 0)});
        }
    }
    std::stable_sort(rows.begin(), rows.end(), [](auto &x, auto &y) { return x.first > y.first; });
    std::stable_sort(cols.begin(), cols.end(), [](auto &x, auto &y) { return x.first > y.first; });
    std::vector<int2> hr;
    std::vector<int4> hc;
    for (auto &x : rows) hr.push_back(x.second);
    for (auto &x : cols) hc.push_back(x.second);
    cudaError_t e = cudaMalloc(&ctx->row_items, sizeof(int2) * hr.size());
    if (e == cudaSuccess) e = cudaMalloc(&ctx->col_items, sizeof(int4) * hc.size());
    if (e == cudaSuccess) e = cudaMalloc(&ctx->counter, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemcpy(ctx->row_items, hr.data(), sizeof(int2) * hr.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->col_items, hc.data(), sizeof(int4) * hc.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(ctx->counter, 0, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = prepare_rows_batch<float>(smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch work lists");
    ctx->nrow_items = (int)hr.size();
    ctx->ncol_items = (int)hc.size();
    ctx->row_smem = smem;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    ctx->row_grid = sms;          // one 512-thread CTA per SM (128 registers)
    ctx->col_grid = 2 * sms;      // column CTAs use fewer registers
    return FCN_OK;
}

// Automatic choice: the work lists pay off when the grids differ and most
// of the batch's points lie in pulses whose own row launch cannot fill the
// GPU (fewer row CTAs than twice the SM count), which a launch per pulse
// would serialise as part-empty launches.  Measured on GB300: 64 uneven
// pulses of Nr 64-256 x Nt 512-1024 run 5.8x faster batched; the 64 pulses
// of Nr 256-2048 x Nt 512-8192 run 6 % faster as tuned per-pulse launches.
// Identical grids always run per-pulse (paired) launches.
bool grids_uneven(const fcn_ctx *ctx) {
    for (auto &pu : ctx->pulses)
        if (pu.g.nr != ctx->pulses[0].g.nr || pu.g.nt != ctx->pulses[0].g.nt) return true;
    return false;
}

bool small_pulses_dominate(const fcn_ctx *ctx) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double small = 0.0, all = 0.0;
    for (auto &pu : ctx->pulses) {
        const int tpr = pu.g.nt >= 16 ? pu.g.nt / 16 : 1;
        const int rpc = tpr >= 256 ? 1 : 256 / tpr;           // rows per CTA of the per-Nt kernels
        const int ctas = (pu.g.nr + rpc - 1) / rpc;
        const double pts = (double)pu.points();
        all += pts;
        if (ctas < 2 * sms) small += pts;
    }
    return small > 0.5 * all;
}

int create_impl(int n, const fcn_grid *grids, const fcn_params *params, int prec, void *stream,
                fcn_ctx **out) {
    if (!out) return fail(nullptr, FCN_ERR_ARG, "out is null");
    *out = nullptr;
    if (n < 1 || !grids || !params) return fail(nullptr, FCN_ERR_ARG, "need n >= 1 grids and params");
    for (int i = 0; i < n; ++i) {
        std::string why;
        int rc = check_grid_params(prec, &grids[i], &params[i], &why);
        if (rc) return fail(nullptr, rc, "pulse " + std::to_string(i) + ": " + why);
    }
    fcn_ctx *ctx = new fcn_ctx();
    ctx->prec = prec;
    ctx->st = (cudaStream_t)stream;
    ctx->pulses.resize(n);
    int rc = FCN_OK;
    auto bail = [&](int code) {
        g_create_error = ctx->err;
        fcn_destroy(ctx);
        return code;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) { cuda_fail(ctx, e, "stream"); return bail(FCN_ERR_CUDA); }
    e = cudaMallocHost(&ctx->host_red, 16 * sizeof(double));
    if (e != cudaSuccess) { cuda_fail(ctx, e, "pinned buffer"); return bail(FCN_ERR_NOMEM); }
    for (int i = 0; i < n && rc == FCN_OK; ++i) {
        Pulse &pu = ctx->pulses[i];
        pu.g = grids[i];
        pu.p = params[i];
        const size_t np = (size_t)pu.points();
        if ((e = cudaMalloc(&pu.field, csize(prec) * np)) != cudaSuccess ||
            (e = cudaMalloc(&pu.rho, rsize(prec) * np)) != cudaSuccess ||
            (e = cudaMalloc(&pu.stats, sizeof(double) * NSTAT * pu.g.nr)) != cudaSuccess ||
            (e = cudaMalloc(&pu.red, sizeof(double) * 16)) != cudaSuccess ||
            (e = cudaMalloc(&pu.rows, sizeof(double) * 2 * pu.g.nr)) != cudaSuccess ||
            (e = cudaMalloc(&pu.err, sizeof(int))) != cudaSuccess) {
            cuda_fail(ctx, e, "device allocation");
            return bail(FCN_ERR_NOMEM);
        }
        cudaMemset(pu.err, 0, sizeof(int));
        cudaMemset(pu.field, 0, csize(prec) * np);
        cudaMemset(pu.rho, 0, rsize(prec) * np);
        cudaMemset(pu.stats, 0, sizeof(double) * NSTAT * pu.g.nr);
        if (prec == FCN_FP64) {
            const cx<double> *tw;
            const double *lo, *hi;
            if ((e = get_twiddles<double>(pu.g.nt, &tw)) != cudaSuccess ||
                (e = get_lohi<double>(pu.g.nr, &lo, &hi, &pu.lo64, &pu.hi64)) != cudaSuccess) {
                cuda_fail(ctx, e, "constant tables");
                return bail(FCN_ERR_CUDA);
            }
            pu.tw = tw; pu.lo = lo; pu.hi = hi;
            if ((e = prepare_rows<double>(pu.g.nt)) != cudaSuccess || (e = prepare_cn<double>()) != cudaSuccess) {
                cuda_fail(ctx, e, "row kernel attributes");
                return bail(FCN_ERR_CUDA);
            }
        } else {
            const cx<float> *tw, *tw1 = nullptr;
            const float *lo, *hi;
            if ((e = get_twiddles<float>(pu.g.nt, &tw)) != cudaSuccess ||
                (pu.g.nt >= 256 && (e = get_twiddles<float>(fft_tag(pu.g.nt, 1), &tw1)) != cudaSuccess) ||
                (e = get_lohi<float>(pu.g.nr, &lo, &hi, &pu.lo64, &pu.hi64)) != cudaSuccess) {
                cuda_fail(ctx, e, "constant tables");
                return bail(FCN_ERR_CUDA);
            }
            pu.tw = tw; pu.tw1 = tw1; pu.lo = lo; pu.hi = hi;
            if ((e = prepare_rows<float>(pu.g.nt)) != cudaSuccess || (e = prepare_cn<float>()) != cudaSuccess) {
                cuda_fail(ctx, e, "row kernel attributes");
                return bail(FCN_ERR_CUDA);
            }
        }
    }
    if (n > 1 && prec == FCN_FP32_MIXED) {
        int rc = setup_batch(ctx);
        if (rc) return bail(rc);
        ctx->batched = ctx->row_items != nullptr && grids_uneven(ctx) && small_pulses_dominate(ctx);
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) { cuda_fail(ctx, e, "init sync"); return bail(FCN_ERR_CUDA); }
    *out = ctx;
    return FCN_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// exported C-ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *fcn_version(void) { return "fcn-gb300 0.1 (sm_103a)"; }

int fcn_create(const fcn_grid *grid, const fcn_params *params, int32_t precision, void *stream,
               fcn_ctx **out) {
    return create_impl(1, grid, params, precision, stream, out);
}

int fcn_create_batch(int32_t n, const fcn_grid *grids, const fcn_params *params, int32_t precision,
                     void *stream, fcn_ctx **out) {
    return create_impl(n, grids, params, precision, stream, out);
}

void fcn_destroy(fcn_ctx *ctx) {
    if (!ctx) return;
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    cudaDeviceSynchronize();
    drop_graphs(ctx, true, 0);
    profile_collect(ctx);
    for (auto &pu : ctx->pulses) {
        cudaFree(pu.field);
        cudaFree(pu.work1);
        cudaFree(pu.work2);
        cudaFree(pu.rho);
        cudaFree(pu.stats);
        cudaFree(pu.red);
        cudaFree(pu.rows);
        cudaFree(pu.stage);
        cudaFree(pu.err);
    }
    for (auto &kv : ctx->tables) cudaFree(kv.second.ptr);
    if (ctx->mlp) cudaFree(ctx->mlp);
    cudaFree(ctx->mlp_io);
    cudaFree(ctx->batch_io);
    if (ctx->host_ctl) cudaFreeHost(ctx->host_ctl);
    for (auto &kv : ctx->batch_args) {
        cudaFree(kv.second.first);
        cudaFree(kv.second.second);
    }
    cudaFree(ctx->row_items);
    cudaFree(ctx->col_items);
    cudaFree(ctx->counter);
    if (ctx->host_red) cudaFreeHost(ctx->host_red);
    for (int b = 0; b < kMaxBranches; ++b) {
        if (ctx->bst[b]) cudaStreamDestroy(ctx->bst[b]);
        if (ctx->join_ev[b]) cudaEventDestroy(ctx->join_ev[b]);
    }
    for (int k = 0; k < 2; ++k) {
        if (ctx->tside[k]) cudaStreamDestroy(ctx->tside[k]);
        if (ctx->tbefore[k]) cudaEventDestroy(ctx->tbefore[k]);
        if (ctx->tready[k]) cudaEventDestroy(ctx->tready[k]);
    }
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    delete ctx;
}

const char *fcn_last_error(const fcn_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

int fcn_set_stream(fcn_ctx *ctx, void *stream) {
    if (!ctx) return FCN_ERR_ARG;
    ctx->st = (cudaStream_t)stream;
    return FCN_OK;
}

int fcn_set_field(fcn_ctx *ctx, int32_t pulse, const double *host) {
    Pulse *pu = get_pulse(ctx, pulse);
    if (!pu || !host) return fail(ctx, FCN_ERR_ARG, "bad pulse index or null buffer");
    const size_t np = (size_t)pu->points();
    if (ctx->prec == FCN_FP64) {
        CK(cudaMemcpyAsync(pu->field, host, 16 * np, cudaMemcpyHostToDevice, ctx->st), "H2D field");
    } else {
        if (!pu->stage) CK(cudaMalloc(&pu->stage, 16 * np), "staging buffer");
        CK(cudaMemcpyAsync(pu->stage, host, 16 * np, cudaMemcpyHostToDevice, ctx->st), "H2D field");
        CK(launch_narrow<float>(pu->stage, (cx<float> *)pu->field, (int64_t)np, ctx->st), "narrow");
    }
    CK(cudaMemsetAsync(pu->stats, 0, sizeof(double) * NSTAT * pu->g.nr, ctx->st), "reset stats");
    CK(cudaMemsetAsync(pu->rho, 0, rsize(ctx->prec) * np, ctx->st), "reset rho");
    pu->z = 0.0;
    pu->steps = pu->rejected = 0;
    pu->dz_next = 0.0;
    pu->has_field = true;
    return FCN_OK;
}

int fcn_set_field_device(fcn_ctx *ctx, int32_t pulse, const void *dev) {
    Pulse *pu = get_pulse(ctx, pulse);
    if (!pu || !dev) return fail(ctx, FCN_ERR_ARG, "bad pulse index or null buffer");
    const size_t np = (size_t)pu->points();
    CK(cudaMemcpyAsync(pu->field, dev, csize(ctx->prec) * np, cudaMemcpyDeviceToDevice, ctx->st), "D2D field");
    CK(cudaMemsetAsync(pu->stats, 0, sizeof(double) * NSTAT * pu->g.nr, ctx->st), "reset stats");
    CK(cudaMemsetAsync(pu->rho, 0, rsize(ctx->prec) * np, ctx->st), "reset rho");
    pu->z = 0.0;
    pu->steps = pu->rejected = 0;
    pu->has_field = true;
    return FCN_OK;
}

// FCN_ERR_CUDA when a kernel of this pulse recorded that a bounded wait gave
// up (the field is then not valid); synchronises the context stream.
// (a launch over several pulses records in the first pulse's flag)
static int check_wait_flag(fcn_ctx *ctx, const Pulse &pu) {
    int h[2] = {0, 0};
    CK(cudaMemcpyAsync(&h[0], pu.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st), "error flag");
    CK(cudaMemcpyAsync(&h[1], ctx->pulses[0].err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st), "error flag");
    CK(cudaStreamSynchronize(ctx->st), "sync");
    if (h[0] || h[1])
        return fail(ctx, FCN_ERR_CUDA, (h[0] | h[1]) & 1 ? "column stage: a bounded wait for a TMA copy gave up"
                                                          : "row stage: a bounded wait for a row copy gave up");
    return FCN_OK;
}

int fcn_get_field(fcn_ctx *ctx, int32_t pulse, double *host) {
    Pulse *pu = get_pulse(ctx, pulse);
    if (!pu || !host) return fail(ctx, FCN_ERR_ARG, "bad pulse index or null buffer");
    const size_t np = (size_t)pu->points();
    if (ctx->prec == FCN_FP64) {
        CK(cudaMemcpyAsync(host, pu->field, 16 * np, cudaMemcpyDeviceToHost, ctx->st), "D2H field");
    } else {
        if (!pu->stage) CK(cudaMalloc(&pu->stage, 16 * np), "staging buffer");
        CK(launch_widen<float>((const cx<float> *)pu->field, pu->stage, (int64_t)np, ctx->st), "widen");
        CK(cudaMemcpyAsync(host, pu->stage, 16 * np, cudaMemcpyDeviceToHost, ctx->st), "D2H field");
    }
    return check_wait_flag(ctx, *pu);
}

int fcn_set_field_c64(fcn_ctx *ctx, int32_t pulse, const float *host) {
    Pulse *pu = get_pulse(ctx, pulse);
    if (!pu || !host) return fail(ctx, FCN_ERR_ARG, "bad pulse index or null buffer");
    const size_t np = (size_t)pu->points();
    if (ctx->prec == FCN_FP32_MIXED) {
        CK(cudaMemcpyAsync(pu->field, host, 8 * np, cudaMemcpyHostToDevice, ctx->st), "H2D field");
    } else {
        if (!pu->stage) CK(cudaMalloc(&pu->stage, 16 * np), "staging buffer");
        CK(cudaMemcpyAsync(pu->stage, host, 8 * np, cudaMemcpyHostToDevice, ctx->st), "H2D field");
        CK(launch_widen<float>((const cx<float> *)pu->stage, (double *)pu->field, (int64_t)np, ctx->st), "widen");
    }
    CK(cudaMemsetAsync(pu->stats, 0, sizeof(double) * NSTAT * pu->g.nr, ctx->st), "reset stats");
    CK(cudaMemsetAsync(pu->rho, 0, rsize(ctx->prec) * np, ctx->st), "reset rho");
    pu->z = 0.0;
    pu->steps = pu->rejected = 0;
    pu->dz_next = 0.0;
    pu->has_field = true;
    return FCN_OK;
}

int fcn_get_field_c64(fcn_ctx *ctx, int32_t pulse, float *host) {
    Pulse *pu = get_pulse(ctx, pulse);
    if (!pu || !host) return fail(ctx, FCN_ERR_ARG, "bad pulse index or null buffer");
    const size_t np = (size_t)pu->points();
    if (ctx->prec == FCN_FP32_MIXED) {
        CK(cudaMemcpyAsync(host, pu->field, 8 * np, cudaMemcpyDeviceToHost, ctx->st), "D2H field");
    } else {
        if (!pu->stage) CK(cudaMalloc(&pu->stage, 16 * np), "staging buffer");
        CK(launch_narrow<float>((const double *)pu->field, (cx<float> *)pu->stage, (int64_t)np, ctx->st), "narrow");
        CK(cudaMemcpyAsync(host, pu->stage, 8 * np, cudaMemcpyDeviceToHost, ctx->st), "D2H field");
    }
    return check_wait_flag(ctx, *pu);
}

int fcn_get_field_device(fcn_ctx *ctx, int32_t pulse, void *dev) {
    Pulse *pu = get_pulse(ctx, pulse);
    if (!pu || !dev) return fail(ctx, FCN_ERR_ARG, "bad pulse index or null buffer");
    CK(cudaMemcpyAsync(dev, pu->field, csize(ctx->prec) * pu->points(), cudaMemcpyDeviceToDevice, ctx->st),
       "D2D field");
    return FCN_OK;
}

int fcn_get_rho(fcn_ctx *ctx, int32_t pulse, double *host) {
    Pulse *pu = get_pulse(ctx, pulse);
    if (!pu || !host) return fail(ctx, FCN_ERR_ARG, "bad pulse index or null buffer");
    const size_t np = (size_t)pu->points();
    if (ctx->prec == FCN_FP64) {
        CK(cudaMemcpyAsync(host, pu->rho, 8 * np, cudaMemcpyDeviceToHost, ctx->st), "D2H rho");
    } else {
        if (!pu->stage) CK(cudaMalloc(&pu->stage, 16 * np), "staging buffer");
        CK(launch_widen_real<float>((const float *)pu->rho, pu->stage, (int64_t)np, ctx->st), "widen rho");
        CK(cudaMemcpyAsync(host, pu->stage, 8 * np, cudaMemcpyDeviceToHost, ctx->st), "D2H rho");
    }
    CK(cudaStreamSynchronize(ctx->st), "sync");
    return FCN_OK;
}

int fcn_step(fcn_ctx *ctx, double dz, int64_t n) {
    if (!ctx) return FCN_ERR_ARG;
    return ctx->prec == FCN_FP64 ? step_impl<double>(ctx, dz, n, true) : step_impl<float>(ctx, dz, n, true);
}

int fcn_step_nograph(fcn_ctx *ctx, double dz, int64_t n) {
    if (!ctx) return FCN_ERR_ARG;
    return ctx->prec == FCN_FP64 ? step_impl<double>(ctx, dz, n, false) : step_impl<float>(ctx, dz, n, false);
}

int fcn_propagate(fcn_ctx *ctx, double z_end, double dz0, double rtol, double dz_min, int32_t max_reject,
                  int32_t controller, fcn_stats *out) {
    if (!ctx) return FCN_ERR_ARG;
    return ctx->prec == FCN_FP64
               ? propagate_impl<double>(ctx, z_end, dz0, rtol, dz_min, max_reject, controller, out)
               : propagate_impl<float>(ctx, z_end, dz0, rtol, dz_min, max_reject, controller, out);
}

int fcn_get_diag(fcn_ctx *ctx, int32_t pulse, fcn_diag *out) {
    Pulse *pu = get_pulse(ctx, pulse);
    if (!pu || !out) return fail(ctx, FCN_ERR_ARG, "bad pulse index or null output");
    const int rc = check_wait_flag(ctx, *pu);
    if (rc) return rc;
    return ctx->prec == FCN_FP64 ? diag_impl<double>(ctx, *pu, out) : diag_impl<float>(ctx, *pu, out);
}

int fcn_get_profiles(fcn_ctx *ctx, int32_t pulse, double *power, double *fluence) {
    Pulse *pu = get_pulse(ctx, pulse);
    if (!pu) return fail(ctx, FCN_ERR_ARG, "bad pulse index");
    const int nr = pu->g.nr, nt = pu->g.nt;
    double *d = nullptr;
    CK(cudaMalloc(&d, sizeof(double) * (nt + nr)), "profile buffer");
    cudaError_t e = ctx->prec == FCN_FP64
        ? launch_profiles<double>((const cx<double> *)pu->field, nr, nt, d, d + nt, ctx->st)
        : launch_profiles<float>((const cx<float> *)pu->field, nr, nt, d, d + nt, ctx->st);
    std::vector<double> h(nt + nr);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, sizeof(double) * (nt + nr), cudaMemcpyDeviceToHost, ctx->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "profiles");
    const Consts c = derive(pu->g, pu->p);
    if (power)
        for (int p = 0; p < nt; ++p) power[p] = 2.0 * kPi * c.dr * c.dr * h[p];
    if (fluence)
        for (int m = 0; m < nr; ++m) fluence[m] = c.dtau * h[nt + m];
    return FCN_OK;
}

int fcn_get_state(fcn_ctx *ctx, int32_t pulse, double state[4]) {
    Pulse *pu = get_pulse(ctx, pulse);
    if (!pu || !state) return fail(ctx, FCN_ERR_ARG, "bad pulse index or null state");
    state[0] = pu->z;
    state[1] = double(pu->steps);
    state[2] = double(pu->rejected);
    state[3] = pu->dz_next;
    return FCN_OK;
}

int fcn_set_state(fcn_ctx *ctx, int32_t pulse, const double state[4]) {
    Pulse *pu = get_pulse(ctx, pulse);
    if (!pu || !state) return fail(ctx, FCN_ERR_ARG, "bad pulse index or null state");
    pu->z = state[0];
    pu->steps = (int64_t)state[1];
    pu->rejected = (int64_t)state[2];
    pu->dz_next = state[3];
    return FCN_OK;
}

int fcn_set_variants(fcn_ctx *ctx, int32_t row_variant, int32_t col_variant) {
    if (!ctx) return FCN_ERR_ARG;
    if (row_variant < -1 || row_variant >= kRowVariants || col_variant < -1 || col_variant >= kColVariants)
        return fail(ctx, FCN_ERR_ARG, "variant out of range");
    CK(cudaStreamSynchronize(ctx->st), "sync");
    ctx->force_row = row_variant;
    ctx->force_col = col_variant;
    ctx->pairs = -1;
    for (auto &pu : ctx->pulses) pu.tuned = false;
    ctx->seq_all = -1;
    drop_graphs(ctx, true, 0);
    return FCN_OK;
}

int fcn_set_batching(fcn_ctx *ctx, int32_t mode) {
    if (!ctx || mode < -1 || mode > 1) return FCN_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->st), "sync");
    const bool possible = ctx->row_items != nullptr;
    if (mode == 1 && !possible)
        return fail(ctx, FCN_ERR_UNSUPPORTED, "work lists need several FP32 pulses with K = 8 and Nt >= 512");
    const bool want = mode == 1 || (mode == -1 && possible && grids_uneven(ctx) && small_pulses_dominate(ctx));
    if (want != ctx->batched) {
        drop_graphs(ctx, true, 0);
        ctx->batched = want;
    }
    return FCN_OK;
}

int fcn_set_pairing(fcn_ctx *ctx, int32_t mode) {
    if (!ctx || mode < -1 || mode > 1) return FCN_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->st), "sync");
    ctx->pair_mode = mode;
    ctx->pairs = -1;
    ctx->seq_all = -1;
    drop_graphs(ctx, true, 0);
    return FCN_OK;
}

int fcn_get_pairing(const fcn_ctx *ctx) { return ctx ? ctx->pairs : FCN_ERR_ARG; }

int fcn_set_sequential_columns(fcn_ctx *ctx, int32_t mode) {
    if (!ctx || mode < -1 || mode > 1 + kSeqShapes) return FCN_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->st), "sync");
    ctx->seq_mode = mode > 1 ? 1 : mode;
    ctx->seq_shape = mode > 1 ? mode - 2 : 0;
    ctx->seq_all = -1;
    drop_graphs(ctx, true, 0);
    return FCN_OK;
}

int fcn_get_sequential_columns(const fcn_ctx *ctx) { return ctx ? ctx->seq_all : FCN_ERR_ARG; }

int fcn_set_graph_branches(fcn_ctx *ctx, int32_t n) {
    if (!ctx) return FCN_ERR_ARG;
    if (n < 1 || n > kMaxBranches) return fail(ctx, FCN_ERR_ARG, "branches must be in 1..8");
    CK(cudaStreamSynchronize(ctx->st), "sync");
    if (!ctx->fork_ev) CK(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming), "fork event");
    for (int b = 0; b < n; ++b) {
        if (!ctx->bst[b]) CK(cudaStreamCreateWithFlags(&ctx->bst[b], cudaStreamNonBlocking), "branch stream");
        if (!ctx->join_ev[b]) CK(cudaEventCreateWithFlags(&ctx->join_ev[b], cudaEventDisableTiming), "join event");
    }
    ctx->branches = n;
    ctx->seq_all = -1;
    drop_graphs(ctx, true, 0);
    return FCN_OK;
}

int fcn_get_graph_branches(const fcn_ctx *ctx) { return ctx ? ctx->branches : FCN_ERR_ARG; }

int fcn_set_multi_launch(fcn_ctx *ctx, int32_t mode) {
    if (!ctx || mode < 0 || mode > 2) return FCN_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->st), "sync");
    if (mode != ctx->multi_mode) {
        ctx->multi_mode = mode;
        ctx->seq_all = -1;
        drop_graphs(ctx, true, 0);
    }
    return FCN_OK;
}

int fcn_get_multi_launch(const fcn_ctx *ctx) { return ctx ? ctx->multi_mode : FCN_ERR_ARG; }

int fcn_get_variants(fcn_ctx *ctx, int32_t pulse, int32_t out[2]) {
    Pulse *pu = get_pulse(ctx, pulse);
    if (!pu || !out) return fail(ctx, FCN_ERR_ARG, "bad pulse index or null output");
    out[0] = pu->tuned ? pu->row_var : -1;
    out[1] = pu->tuned ? pu->col_var : -1;
    return FCN_OK;
}

int fcn_profile_enable(fcn_ctx *ctx, int32_t on) {
    if (!ctx) return FCN_ERR_ARG;
    if (on < 0 || on > 2) return fail(ctx, FCN_ERR_ARG, "profiling mode must be 0, 1 or 2");
    CK(cudaStreamSynchronize(ctx->st), "profile sync");
    profile_collect(ctx);
    ctx->profiling = on;
    return FCN_OK;
}

int fcn_profile_read(fcn_ctx *ctx, double *ms, int64_t *count, int32_t reset) {
    if (!ctx || !ms || !count) return FCN_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->st), "profile sync");
    profile_collect(ctx);
    for (int k = 0; k < FCN_PROF_KINDS; ++k) {
        ms[k] = ctx->prof_ms[k];
        count[k] = ctx->prof_n[k];
        if (reset) { ctx->prof_ms[k] = 0; ctx->prof_n[k] = 0; }
    }
    return FCN_OK;
}

int fcn_mlp_set_log(fcn_ctx *ctx, float *host_buf, int64_t capacity) {
    if (!ctx || capacity < 0 || (capacity > 0 && !host_buf)) return FCN_ERR_ARG;
    ctx->log_buf = capacity > 0 ? host_buf : nullptr;
    ctx->log_cap = capacity;
    ctx->log_n = 0;
    return FCN_OK;
}

int64_t fcn_mlp_log_count(const fcn_ctx *ctx) { return ctx ? ctx->log_n : -1; }

// Gradient of the mean squared error of the MLP (BF16 weights, FP32
// accumulation) over n samples; stateless, for checking the training kernels.
int fcn_mlp_loss_grad(const float *params, const float *x, const float *y, int32_t n, float *loss,
                      float *grad) {
    fcn_ctx *ctx = nullptr;
    if (!params || !x || !y || n < 1 || !loss || !grad) return fail(nullptr, FCN_ERR_ARG, "bad MLP arguments");
    const int np = mlp_nparam();
    float *dW = nullptr, *dX = nullptr, *dY = nullptr, *dP = nullptr, *dG = nullptr, *dL = nullptr;
    int *dI = nullptr;
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    cudaError_t e = cudaMalloc(&dW, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&dX, sizeof(float) * 6 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&dY, sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&dI, sizeof(int) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&dP, sizeof(float) * 64 * (np + 1));
    if (e == cudaSuccess) e = cudaMalloc(&dG, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&dL, sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(dW, params, sizeof(float) * np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dX, x, sizeof(float) * 6 * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dY, y, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dI, idx.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_mlp_grad(dW, dX, dY, dI, n, dP, 64, dG, dL, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(grad, dG, sizeof(float) * np, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(loss, dL, sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(dW); cudaFree(dX); cudaFree(dY); cudaFree(dI); cudaFree(dP); cudaFree(dG); cudaFree(dL);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "MLP gradient");
    return FCN_OK;
}

// Trains the context's MLP (initialised from the seed if no weights were
// set) with Adam on minibatches of a seeded permutation of the n samples.
int fcn_mlp_train(fcn_ctx *ctx, const float *x, const float *y, int32_t n, int32_t epochs, int32_t batch,
                  float lr, uint64_t seed, float *final_loss) {
    if (!ctx || !x || !y || n < 1 || epochs < 0 || batch < 1 || !(lr > 0)) return FCN_ERR_ARG;
    const int np = mlp_nparam();
    if (!ctx->mlp) CK(cudaMalloc(&ctx->mlp, sizeof(float) * np), "mlp weights");
    uint64_t rs = seed * 6364136223846793005ull + 1442695040888963407ull;
    auto rnd = [&]() {   // splitmix64 -> uniform [0, 1)
        rs += 0x9E3779B97F4A7C15ull;
        uint64_t z = rs;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    if (!ctx->has_mlp) {
        // uniform +-sqrt(6/(fan_in+fan_out)) weights, zero biases
        std::vector<float> w(np, 0.f);
        auto fill = [&](int off, int cnt, int fi, int fo) {
            const double a = std::sqrt(6.0 / (fi + fo));
            for (int i = 0; i < cnt; ++i) w[off + i] = (float)((2.0 * rnd() - 1.0) * a);
        };
        fill(0, 64 * 6, 6, 64);
        fill(64 * 6 + 64, 64 * 64, 64, 64);
        fill(64 * 6 + 64 + 64 * 64 + 64, 64, 64, 1);
        CK(cudaMemcpy(ctx->mlp, w.data(), sizeof(float) * np, cudaMemcpyHostToDevice), "mlp init");
        ctx->has_mlp = true;
    }
    float *dX = nullptr, *dY = nullptr, *dP = nullptr, *dG = nullptr, *dL = nullptr, *dm = nullptr, *dv = nullptr;
    int *dI = nullptr;
    cudaError_t e = cudaMalloc(&dX, sizeof(float) * 6 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&dY, sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&dI, sizeof(int) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&dP, sizeof(float) * 64 * (np + 1));
    if (e == cudaSuccess) e = cudaMalloc(&dG, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&dL, sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dm, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&dv, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMemset(dm, 0, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMemset(dv, 0, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMemcpy(dX, x, sizeof(float) * 6 * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dY, y, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice);
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    int t = 0;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        for (int i = n - 1; i > 0; --i) {   // Fisher-Yates with the seeded generator
            const int j = (int)(rnd() * (i + 1));
            std::swap(idx[i], idx[j]);
        }
        e = cudaMemcpy(dI, idx.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice);
        for (int b0 = 0; b0 < n && e == cudaSuccess; b0 += batch) {
            const int nb = std::min(batch, n - b0);
            e = launch_mlp_grad(ctx->mlp, dX, dY, dI + b0, nb, dP, 64, dG, dL, ctx->st);
            if (e == cudaSuccess) e = launch_mlp_adam(ctx->mlp, dm, dv, dG, lr, ++t, ctx->st);
        }
    }
    if (e == cudaSuccess && final_loss) {
        for (int i = 0; i < n; ++i) idx[i] = i;
        e = cudaMemcpy(dI, idx.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = launch_mlp_grad(ctx->mlp, dX, dY, dI, n, dP, 64, dG, dL, ctx->st);
        if (e == cudaSuccess) e = cudaMemcpy(final_loss, dL, sizeof(float), cudaMemcpyDeviceToHost);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    cudaFree(dX); cudaFree(dY); cudaFree(dI); cudaFree(dP); cudaFree(dG); cudaFree(dL); cudaFree(dm); cudaFree(dv);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "MLP training");
    return FCN_OK;
}

int fcn_mlp_set(fcn_ctx *ctx, const float *host) {
    if (!ctx || !host) return FCN_ERR_ARG;
    if (!ctx->mlp) CK(cudaMalloc(&ctx->mlp, sizeof(float) * FCN_MLP_NPARAM), "mlp weights");
    CK(cudaMemcpy(ctx->mlp, host, sizeof(float) * FCN_MLP_NPARAM, cudaMemcpyHostToDevice), "mlp copy");
    ctx->has_mlp = true;
    return FCN_OK;
}

int fcn_mlp_get(fcn_ctx *ctx, float *host) {
    if (!ctx || !host) return FCN_ERR_ARG;
    if (!ctx->has_mlp) return fail(ctx, FCN_ERR_STATE, "no MLP weights loaded");
    CK(cudaMemcpy(host, ctx->mlp, sizeof(float) * FCN_MLP_NPARAM, cudaMemcpyDeviceToHost), "mlp copy");
    return FCN_OK;
}

// ---- stateless device operations ----

int fcn_op_rows(const fcn_grid *grid, const fcn_params *params, int32_t precision, int32_t ops,
                double dz_half, void *field, void *rho, void *stream) {
    std::string why;
    int rc = check_grid_params(precision, grid, params, &why);
    fcn_ctx *ctx = nullptr;
    if (rc) return fail(nullptr, rc, why);
    if (!field || (ops & ~31) || ((ops & FCN_OP_RHO) && !rho) || !std::isfinite(dz_half))
        return fail(nullptr, FCN_ERR_ARG, "bad field/rho pointer, ops or dz_half");
    const cudaStream_t st = (cudaStream_t)stream;
    if (precision == FCN_FP64) {
        RowArgs<double> a;
        const cx<double> *tw;
        CK(get_twiddles<double>(grid->nt, &tw), "twiddles");
        CK(prepare_rows<double>(grid->nt), "row kernel attributes");
        a.field = (cx<double> *)field; a.tw = tw; a.rho = (double *)rho; a.stats = nullptr;
        a.nr = grid->nr; a.nt = grid->nt; a.ops = ops; a.variant = 0; a.nl = nl_coef<double>(*grid, *params, dz_half);
        CK(launch_rows<double>(a, grid->nt, st), "row stage");
    } else {
        RowArgs<float> a;
        const cx<float> *tw;
        CK(get_twiddles<float>(grid->nt, &tw), "twiddles");
        CK(prepare_rows<float>(grid->nt), "row kernel attributes");
        a.field = (cx<float> *)field; a.tw = tw; a.rho = (float *)rho; a.stats = nullptr;
        a.nr = grid->nr; a.nt = grid->nt; a.ops = ops; a.variant = 0; a.nl = nl_coef<float>(*grid, *params, dz_half);
        CK(launch_rows<float>(a, grid->nt, st), "row stage");
    }
    return FCN_OK;
}

int64_t fcn_cn_table_entries(const fcn_grid *grid) {
    if (!grid || grid->nr < 1 || grid->nt < 2) return 0;
    return (int64_t)grid->nr * (grid->nt / 2 + 1);
}

int fcn_op_cn_table(const fcn_grid *grid, const fcn_params *params, int32_t precision, double dz,
                    void *table, void *stream) {
    std::string why;
    int rc = check_grid_params(precision, grid, params, &why);
    fcn_ctx *ctx = nullptr;
    if (rc) return fail(nullptr, rc, why);
    if (!table || !(dz > 0) || !std::isfinite(dz)) return fail(nullptr, FCN_ERR_ARG, "bad table pointer or dz");
    TableArgs ta;
    ta.nr = grid->nr;
    ta.nt = grid->nt;
    cn_coefs(*grid, *params, dz, &ta.s, &ta.dk);
    const double *lo64, *hi64;
    if (precision == FCN_FP64) {
        const double *lo, *hi;
        CK(get_lohi<double>(grid->nr, &lo, &hi, &lo64, &hi64), "radial tables");
        ta.lo = lo64; ta.hi = hi64;
        CK(launch_cn_table<double>(ta, (cx<double> *)table, (cudaStream_t)stream), "table kernel");
    } else {
        const float *lo, *hi;
        CK(get_lohi<float>(grid->nr, &lo, &hi, &lo64, &hi64), "radial tables");
        ta.lo = lo64; ta.hi = hi64;
        CK(launch_cn_table<float>(ta, (cx<float> *)table, (cudaStream_t)stream), "table kernel");
    }
    return FCN_OK;
}

int fcn_op_cn(const fcn_grid *grid, const fcn_params *params, int32_t precision, double dz,
              const void *table, void *field, void *stream) {
    std::string why;
    int rc = check_grid_params(precision, grid, params, &why);
    fcn_ctx *ctx = nullptr;
    if (rc) return fail(nullptr, rc, why);
    if (!table || !field || !(dz > 0) || !std::isfinite(dz)) return fail(nullptr, FCN_ERR_ARG, "bad pointers or dz");
    double s, dk, disp;
    cn_coefs(*grid, *params, dz, &s, &dk, &disp);
    const double *lo64, *hi64;
    if (precision == FCN_FP64) {
        const double *lo, *hi;
        CK(get_lohi<double>(grid->nr, &lo, &hi, &lo64, &hi64), "radial tables");
        ColArgs<double> a;
        a.field = (cx<double> *)field; a.invden = (const cx<double> *)table; a.lo = lo; a.hi = hi;
        a.nr = grid->nr; a.nt = grid->nt; a.s = s; a.dk = dk; a.disp = disp; a.variant = 0;
        CK(launch_cn<double>(a, (cudaStream_t)stream), "column stage");
    } else {
        const float *lo, *hi;
        CK(get_lohi<float>(grid->nr, &lo, &hi, &lo64, &hi64), "radial tables");
        ColArgs<float> a;
        a.field = (cx<float> *)field; a.invden = (const cx<float> *)table; a.lo = lo; a.hi = hi;
        a.nr = grid->nr; a.nt = grid->nt; a.s = float(s); a.dk = float(dk); a.disp = disp; a.variant = 0;
        CK(launch_cn<float>(a, (cudaStream_t)stream), "column stage");
    }
    return FCN_OK;
}

}  // extern "C"
