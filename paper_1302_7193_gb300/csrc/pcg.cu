// C-ABI implementation of the GB300 line-preconditioned CG solver.
//
// Host side: builds the operator tables of the finite-volume scheme
// (Section 3.1: per-level profiles shared by every column, per-column metric
// terms), owns the device workspace, and drives Algorithm 1 (Section 4.3) as
// CUDA graphs of `passes_per_launch` pairs of fused sweeps.  All scalars of
// the iteration live on the device; the host only polls the per-rhs `done`
// flags between graph launches (two launches are kept in flight so the GPU
// never waits for the poll).
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "../../include/pcg.h"
#include "kernels.cuh"
#include "multigrid.cuh"
#include "single_reduction.cuh"
#include "serve_kernels.cuh"

using pcg::BX;
using pcg::BY;
using pcg::OpView;
using pcg::SolveState;

namespace {

thread_local std::string g_create_error = "no error";
// text that pcg_last_error(NULL) returns when it is not g_create_error (set by
// the allocation-free entry point, cleared by every other null-handle failure)
thread_local const char* g_null_error = nullptr;

struct DevTables {
    void* base = nullptr;       // one allocation for all tables of one precision
    void* mass = nullptr;
    void* wv = nullptr;
    void* dk = nullptr;
    void* area = nullptr;
    void* mue = nullptr;
    void* mun = nullptr;
    void* fg = nullptr;
    void* fe = nullptr;
    void* fc = nullptr;
    void* amass = nullptr;      // FP64 only: [rows][nz] area-folded level tables, or null
    void* awv = nullptr;
};

}  // namespace

struct pcg_ctx {
    int geometry = 0, nx = 0, ny = 0, nz = 0, nrhs = 1;
    long long plane = 0, vol = 0, ntot = 0;
    int periodic_y = 1;
    int cls_mode = 0, ncls = 1;
    int precision = PCG_FP64;
    double inner_tol = 1e-5;
    int inner_maxit = 20000, max_outer = 16, ppl = 16;
    int trace = 0;                        // PCG_TRACE=1: print the refinement history to stderr
    double total_mass = 0.0;              // sum over cells of |T| a_k = sum(A 1) per right-hand side
    cudaStream_t stream = nullptr;        // user stream (may be the default stream)
    cudaStream_t cap_stream = nullptr;    // private stream used only for graph capture

    DevTables t64, t32;

    // workspace
    double *u64 = nullptr, *r64 = nullptr, *z64 = nullptr, *p64 = nullptr, *q64 = nullptr;
    float *u32 = nullptr, *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr;
    // tensor maps of the FP32 u, p, q (own tile) and z (tile with halo) for the TMA SpMV sweep
    CUtensorMap tm_u, tm_p, tm_q, tm_z;
    bool tma_ready = false;
    int tma_by = 4;                       // rows of the TMA SpMV tile (4; PCG_TMA_BY=8 for 8)
    // ... and of r, q for the TMA preconditioner sweep (box 32 x prec_R x nch * lz_a)
    CUtensorMap tm_pr, tm_pq;
    // ... and of u, p, q, z for the pipelined TMA SpMV sweep (8-level chunks)
    CUtensorMap tm2_u, tm2_p, tm2_q, tm2_z;
    bool tma2_ready = false;
    int spmv2_G = 1, spmv2_nch = 1, spmv2_gx = 1, spmv2_gy = 1;
    int prec32 = 0;                       // FP32 preconditioner sweep: 0 column/chunked, 2 TMA pipeline
    bool prec_tma_ready = false;
    int prec_R = 1, prec_gx = 1, prec_items = 0, prec_G = 1;
    int prec_generic = 0;                 // 1: the TMA preconditioner sweep without per-level tables
    int pdl = 1;                          // FP32 TMA sweeps launched with programmatic dependencies (PCG_PDL=0: off)
    dim3 grid_t, block_t;
    int nblk_t = 0;
    double *hb = nullptr, *hx = nullptr;  // device staging for pcg_solve_host
    SolveState* st = nullptr;              // [nrhs] outer / FP64 state
    SolveState* st_in = nullptr;           // [nrhs] inner FP32 state
    SolveState* h_st = nullptr;            // pinned [2][nrhs] poll slots
    int* d_active = nullptr;               // [nrhs]
    double* partials = nullptr;            // [nrhs][nblocks][4]
    unsigned* counters = nullptr;          // [nrhs]
    int nblocks = 0;
    dim3 grid, block;
    // chunked sweeps (levels split across threads): launch shapes
    int chunked32 = 0, chunked64 = 0, lz_a = 16, lz_b = 16, nch_b = 1;
    int spmv32 = 0, spmv64 = 0;          // SpMV sweep variant: 0 per column, 1 chunked, 3 TMA,
                                          // 4 persistent two-stage TMA
    dim3 grid_a, block_a, grid_b, block_b;
    int nblk_a = 0, nblk_b = 0;
    dim3 grid_c, block_c;                 // one-thread-per-column sweeps: 32 x by column tiles
    int nblk_c = 0;
    int ksplit = 1;                       // one-thread-per-column SpMV sweep: parts of each column
    // multigrid preconditioner (PCG_PREC_MULTIGRID): coarse levels 1..L-1
    struct MGLevel {
        pcg_ctx* h = nullptr;             // the level's own handle (tables, factors, launch shapes)
        double *r = nullptr, *z = nullptr, *t = nullptr;   // right-hand side, correction, scratch (FP64 cycle)
        float *rf = nullptr, *zf = nullptr, *tf = nullptr; // the same for an FP32 cycle
    };
    int precond = PCG_PREC_LINE;
    std::vector<MGLevel> mg;
    double* mg_t0 = nullptr;              // scratch of level 0
    float *mg_r0f = nullptr, *mg_z0f = nullptr, *mg_t0f = nullptr;   // level 0 of an FP32 cycle
    bool mg_f32 = false;                  // PCG_PREC_MULTIGRID_F32: the V-cycle in FP32
    SolveState* mg_free = nullptr;        // all-active states for a V-cycle outside a solve
    int mg_nu = 1, mg_coarse = 8;
    long long mg_resid_threads = 524288;  // k_mg_resid splits columns until this many threads run
    long long mg_quad = 16384;            // FP32 residuals on float4 quads of row pairs on levels of at least this many columns (0: none)
    long long mg_tail_cols = 4096;        // levels of at most this many columns may run in k_mg_tail (0: none)
    long long mg_tail_smem = 200 * 1024;  // dynamic shared memory k_mg_tail may use for the levels' vectors
    // PCG_ALG_SINGLE_REDUCTION: one k_sweep_sr per pass; r, s (q64), w double-buffered
    bool alg_sr = false;
    dim3 grid_sr;
    int nblk_sr = 0;
    double *r64b = nullptr, *s64b = nullptr, *w64a = nullptr, *w64b = nullptr;
    float *r32b = nullptr, *s32b = nullptr, *w32a = nullptr, *w32b = nullptr;   // the mixed form's inner solve
    cudaGraphExec_t graph_sr = nullptr, graph_sr32 = nullptr;
    double mg_omega = 0.8;
    int kernels_per_pass = 2;             // kernel launches in one Algorithm-1 pass of the graphs
    int spmv_pipe = 1;                    // FP64 SpMV sweep with u, p, q loads issued ahead (PCG_SPMV_PIPE=0: plain)

    cudaGraphExec_t graph64 = nullptr, graph32 = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};

    size_t bytes = 0;
    long long launches = 0;
    std::vector<pcg_stats_t> rhs_stats;
    std::string err = "no error";

    OpView<double> view64() const { return view<double>(t64); }
    OpView<float> view32() const { return view<float>(t32); }

    template <typename T>
    OpView<T> view(const DevTables& t) const {
        OpView<T> v;
        v.nx = nx;
        v.ny = ny;
        v.nz = nz;
        v.plane = plane;
        v.vol = vol;
        v.mass = (const T*)t.mass;
        v.wv = (const T*)t.wv;
        v.dk = (const T*)t.dk;
        v.area = (const T*)t.area;
        v.mue = (const T*)t.mue;
        v.mun = (const T*)t.mun;
        v.periodic_y = periodic_y;
        v.fg = (const T*)t.fg;
        v.fe = (const T*)t.fe;
        v.fc = (const T*)t.fc;
        v.cls_mode = cls_mode;
        v.ncls = ncls;
        v.area_percol = geometry == PCG_GEOM_CUBED_PANEL ? 1 : 0;
        v.amass = (const T*)t.amass;
        v.awv = (const T*)t.awv;
        v.arow_step = geometry == PCG_GEOM_LATLON ? 1 : 0;
        return v;
    }
};

namespace {

int fail(pcg_t h, int code, const std::string& msg) {
    if (h) {
        h->err = msg;
    } else {
        g_create_error = msg;
        g_null_error = nullptr;
    }
    return code;
}

#define PCG_CK(h, call)                                                                       \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            int code_ = (e_ == cudaErrorMemoryAllocation) ? PCG_ERR_OOM : PCG_ERR_CUDA;       \
            return fail(h, code_, std::string(#call) + ": " + cudaGetErrorString(e_));        \
        }                                                                                     \
    } while (0)

template <typename T>
int dmalloc(pcg_t h, T** p, size_t count) {
    size_t b = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void**)p, b);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(h, e == cudaErrorMemoryAllocation ? PCG_ERR_OOM : PCG_ERR_CUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->bytes += b;
    return PCG_OK;
}

// Host computation of the operator tables (Section 3.1; Section 4.2 stores
// per-level vectors once and per-column metric terms once per column).
struct HostTables {
    std::vector<double> mass, wv, dk, area, mue, mun;
};

// Where the tables go: n_z values each of mass, wv, dk; area_len values of
// area (n_y, or n_x n_y for the panel); n_x n_y values each of mue, mun.
struct TableOut {
    double *mass, *wv, *dk, *area, *mue, *mun;
};

// Number of area values of a geometry: one per latitude (or box) row, one
// per column on the panel.
size_t table_area_len(const pcg_grid_t* g) {
    return g->geometry == PCG_GEOM_CUBED_PANEL ? (size_t)g->n_x * g->n_y : (size_t)g->n_y;
}

// Fill the tables of grid g and coefficients c into caller-supplied arrays.
// Allocates nothing; on invalid input returns PCG_ERR_INVALID_ARG with a
// static message in *err.  total_mass = sum over cells of |T| a_k.
int tables_into(const pcg_grid_t* g, const pcg_coeffs_t* c, const TableOut& t, const char** err,
                double* total_mass) {
    auto bad = [&](const char* m) { *err = m; return PCG_ERR_INVALID_ARG; };
    const int nx = g->n_x, ny = g->n_y, nz = g->n_z;
    const double* z = g->z_iface;
    const double* beta = c->beta_iface;
    for (int k = 0; k <= nz; ++k) {
        if (!std::isfinite(z[k]) || !std::isfinite(beta[k])) return bad("non-finite z_iface or beta_iface");
        if (k > 0 && !(z[k] > z[k - 1])) return bad("z_iface must be strictly increasing");
    }
    auto centre = [&](int k) { return 0.5 * (z[k] + z[k + 1]); };
    const size_t nxy = (size_t)nx * ny;
    if (g->geometry == PCG_GEOM_BOX) {
        if (!(g->lx > 0.0) || !(g->ly > 0.0)) return bad("box extents must be positive");
        const double hx = g->lx / nx, hy = g->ly / ny;
        for (int k = 0; k < nz; ++k) {
            const double dz = z[k + 1] - z[k];
            t.mass[k] = c->lambda2 * dz;
            t.dk[k] = dz;
            t.wv[k] = (k + 1 < nz) ? beta[k + 1] / (centre(k + 1) - centre(k)) : 0.0;
        }
        for (int j = 0; j < ny; ++j) t.area[j] = hx * hy;
        for (size_t idx = 0; idx < nxy; ++idx) {
            const double ae = c->alpha_e ? c->alpha_e[idx] : 1.0;
            const double an = c->alpha_n ? c->alpha_n[idx] : 1.0;
            t.mue[idx] = ae * (hy / hx);
            t.mun[idx] = an * (hx / hy);
        }
    } else if (g->geometry == PCG_GEOM_LATLON) {
        const double pi = 3.14159265358979323846;
        if (!(g->lat0 > -0.5 * pi && g->lat1 < 0.5 * pi && g->lat0 < g->lat1))
            return bad("latitude band must satisfy -pi/2 < lat0 < lat1 < pi/2");
        const double dlon = 2.0 * pi / nx, dlat = (g->lat1 - g->lat0) / ny;
        for (int k = 0; k < nz; ++k) {
            // shell volume per unit solid angle, (r1^3 - r0^3)/3 without cancellation
            const double r0 = z[k], r1 = z[k + 1];
            t.mass[k] = c->lambda2 * ((r1 - r0) * (r1 * r1 + r1 * r0 + r0 * r0)) / 3.0;
            t.dk[k] = r1 - r0;
            t.wv[k] = (k + 1 < nz) ? beta[k + 1] * r1 * r1 / (centre(k + 1) - centre(k)) : 0.0;
        }
        for (int j = 0; j < ny; ++j) {
            const double ln = g->lat0 + (j + 1) * dlat, lc = g->lat0 + (j + 0.5) * dlat;
            // dlon (sin ln - sin ls) written as 2 dlon cos(lc) sin(dlat/2): no cancellation
            t.area[j] = dlon * 2.0 * std::cos(lc) * std::sin(0.5 * dlat);
            for (int i = 0; i < nx; ++i) {
                const size_t idx = (size_t)j * nx + i;
                const double ae = c->alpha_e ? c->alpha_e[idx] : 1.0;
                const double an = c->alpha_n ? c->alpha_n[idx] : 1.0;
                t.mue[idx] = ae * dlat / (std::cos(lc) * dlon);
                t.mun[idx] = (j + 1 < ny) ? an * std::cos(ln) * dlon / dlat : 0.0;
            }
        }
    } else if (g->geometry == PCG_GEOM_CUBED_PANEL) {
        // equidistant gnomonic panel: tangent-plane cell [x_i, x_i+1] x [y_j, y_j+1] mapped by
        // P(x, y) = (1, x, y)/|(1, x, y)|.  Area = solid angle of two spherical triangles by Van
        // Oosterom and Strackee's formula for unnormalised vertices, face weight = alpha (edge
        // arc)/(centre arc); every small quantity comes from exact coordinate differences.
        auto nrm = [](double x, double y) { return std::sqrt(1.0 + x * x + y * y); };
        auto arc_same_y = [](double x1, double x2, double y) {
            return std::atan2(std::fabs(x2 - x1) * std::sqrt(1.0 + y * y), 1.0 + x1 * x2 + y * y);
        };
        auto arc_same_x = [](double x, double y1, double y2) {
            return std::atan2(std::fabs(y2 - y1) * std::sqrt(1.0 + x * x), 1.0 + x * x + y1 * y2);
        };
        auto tri = [&](double xa, double ya, double xb, double yb, double xc_, double yc_) {
            const double det = std::fabs((xb - xa) * (yc_ - ya) - (xc_ - xa) * (yb - ya));
            const double na = nrm(xa, ya), nb = nrm(xb, yb), nc = nrm(xc_, yc_);
            const double ab = 1.0 + xa * xb + ya * yb, bc = 1.0 + xb * xc_ + yb * yc_, ca = 1.0 + xc_ * xa + yc_ * ya;
            return 2.0 * std::atan2(det, na * nb * nc + ab * nc + bc * na + ca * nb);
        };
        for (int k = 0; k < nz; ++k) {
            const double r0 = z[k], r1 = z[k + 1];
            t.mass[k] = c->lambda2 * ((r1 - r0) * (r1 * r1 + r1 * r0 + r0 * r0)) / 3.0;
            t.dk[k] = r1 - r0;
            t.wv[k] = (k + 1 < nz) ? beta[k + 1] * r1 * r1 / (centre(k + 1) - centre(k)) : 0.0;
        }
        auto xf = [&](int i) { return -1.0 + 2.0 * i / nx; };
        auto yf = [&](int j) { return -1.0 + 2.0 * j / ny; };
        auto xc = [&](int i) { return 0.5 * (xf(i) + xf(i + 1)); };
        auto yc = [&](int j) { return 0.5 * (yf(j) + yf(j + 1)); };
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                const size_t idx = (size_t)j * nx + i;
                const double x0 = xf(i), x1 = xf(i + 1), y0 = yf(j), y1 = yf(j + 1);
                t.area[idx] = tri(x0, y0, x1, y0, x1, y1) + tri(x0, y0, x1, y1, x0, y1);
                const double ae = c->alpha_e ? c->alpha_e[idx] : 1.0;
                const double an = c->alpha_n ? c->alpha_n[idx] : 1.0;
                t.mue[idx] = (i + 1 < nx) ? ae * (arc_same_x(x1, y0, y1) / arc_same_y(xc(i), xc(i + 1), yc(j))) : 0.0;
                t.mun[idx] = (j + 1 < ny) ? an * (arc_same_y(x0, x1, y1) / arc_same_x(xc(i), yc(j), yc(j + 1))) : 0.0;
            }
        }
    } else {
        return bad("unknown geometry");
    }
    // sum over all cells of |T_j| a_k = sum_i (A 1)_i, the Galerkin coarse operator on the constant vector
    const size_t na = table_area_len(g);
    double sa = 0.0, sm = 0.0;
    for (size_t j = 0; j < na; ++j) sa += t.area[j];
    for (int k = 0; k < nz; ++k) sm += t.mass[k];
    *total_mass = (na == (size_t)ny ? (double)nx : 1.0) * sa * sm;
    return PCG_OK;
}

int build_tables_core(const pcg_grid_t* g, const pcg_coeffs_t* c, HostTables& t, std::string& err,
                      double& total_mass) {
    const int nz = g->n_z;
    const size_t nxy = (size_t)g->n_x * g->n_y;
    t.mass.assign(nz, 0.0);
    t.wv.assign(nz, 0.0);
    t.dk.assign(nz, 0.0);
    t.area.assign(table_area_len(g), 0.0);
    t.mue.assign(nxy, 0.0);
    t.mun.assign(nxy, 0.0);
    const char* msg = nullptr;
    const int rc = tables_into(g, c, TableOut{t.mass.data(), t.wv.data(), t.dk.data(), t.area.data(), t.mue.data(),
                                              t.mun.data()}, &msg, &total_mass);
    if (rc) err = msg;
    return rc;
}

int build_tables(pcg_t h, const pcg_grid_t* g, const pcg_coeffs_t* c, HostTables& t) {
    std::string err;
    const int rc = build_tables_core(g, c, t, err, h->total_mass);
    if (rc) return fail(h, rc, err);
    return PCG_OK;
}

int upload_tables(pcg_t h, const HostTables& t) {
    const size_t nz = h->nz, ny = t.area.size(), nxy = (size_t)h->nx * h->ny, nf = (size_t)nz * h->ncls;
    // area-folded level tables for the FP64 SpMV sweep: one row (box), one per
    // latitude row (latlon), none when the area varies per column (panel)
    const size_t frows = h->geometry == PCG_GEOM_BOX ? 1 : (h->geometry == PCG_GEOM_LATLON ? (size_t)h->ny : 0);
    const size_t n64 = 3 * nz + ny + 2 * nxy + 3 * nf + 2 * frows * nz;
    double* b64 = nullptr;
    float* b32 = nullptr;
    int rc = dmalloc(h, &b64, n64);
    if (rc) return rc;
    rc = dmalloc(h, &b32, n64);
    if (rc) return rc;
    h->t64.base = b64;
    h->t32.base = b32;
    size_t off = 0;
    auto carve = [&](size_t n, void*& p64, void*& p32) {
        p64 = b64 + off;
        p32 = b32 + off;
        off += n;
    };
    carve(nz, h->t64.mass, h->t32.mass);
    carve(nz, h->t64.wv, h->t32.wv);
    carve(nz, h->t64.dk, h->t32.dk);
    carve(ny, h->t64.area, h->t32.area);
    carve(nxy, h->t64.mue, h->t32.mue);
    carve(nxy, h->t64.mun, h->t32.mun);
    carve(nf, h->t64.fg, h->t32.fg);
    carve(nf, h->t64.fe, h->t32.fe);
    carve(nf, h->t64.fc, h->t32.fc);
    void *am32 = nullptr, *aw32 = nullptr;
    if (frows) {
        carve(frows * nz, h->t64.amass, am32);
        carve(frows * nz, h->t64.awv, aw32);
    }
    cudaStream_t s = h->stream;
    PCG_CK(h, cudaMemcpyAsync(h->t64.mass, t.mass.data(), nz * 8, cudaMemcpyHostToDevice, s));
    PCG_CK(h, cudaMemcpyAsync(h->t64.wv, t.wv.data(), nz * 8, cudaMemcpyHostToDevice, s));
    PCG_CK(h, cudaMemcpyAsync(h->t64.dk, t.dk.data(), nz * 8, cudaMemcpyHostToDevice, s));
    PCG_CK(h, cudaMemcpyAsync(h->t64.area, t.area.data(), ny * 8, cudaMemcpyHostToDevice, s));
    PCG_CK(h, cudaMemcpyAsync(h->t64.mue, t.mue.data(), nxy * 8, cudaMemcpyHostToDevice, s));
    PCG_CK(h, cudaMemcpyAsync(h->t64.mun, t.mun.data(), nxy * 8, cudaMemcpyHostToDevice, s));
    if (frows) {
        std::vector<double> fold(2 * frows * nz);
        for (size_t j = 0; j < frows; ++j)
            for (size_t k = 0; k < nz; ++k) {
                fold[j * nz + k] = t.area[j] * t.mass[k];
                fold[(frows + j) * nz + k] = t.area[j] * t.wv[k];
            }
        // pageable source: the copy has consumed it when the call returns
        PCG_CK(h, cudaMemcpyAsync(h->t64.amass, fold.data(), 2 * frows * nz * 8, cudaMemcpyHostToDevice, s));
    }
    // Thomas factors of every class, in FP64 on the device
    const OpView<double> v = h->view64();
    pcg::k_factors<<<(h->ncls + 127) / 128, 128, 0, s>>>(v, (double*)h->t64.fg, (double*)h->t64.fe,
                                                         (double*)h->t64.fc);
    PCG_CK(h, cudaGetLastError());
    const long long nconv = (long long)n64;
    pcg::k_to_float<<<1024, 256, 0, s>>>(b64, b32, nconv);
    PCG_CK(h, cudaGetLastError());
    PCG_CK(h, cudaStreamSynchronize(s));
    return PCG_OK;
}

int ensure_ws64(pcg_t h) {
    if (h->u64) return PCG_OK;
    int rc;
    for (double** p : {&h->u64, &h->r64, &h->z64, &h->p64, &h->q64})
        if ((rc = dmalloc(h, p, (size_t)h->ntot))) return rc;
    return PCG_OK;
}

// PCG_ALG_SINGLE_REDUCTION: the second buffers of r and s, both of w (in the
// precision of the iteration), and the shared-memory limit of its sweep
// (n_z x 108 values)
int ensure_ws_sr(pcg_t h, bool f32) {
    int rc;
    if (f32) {
        if (h->w32b) return PCG_OK;
        for (float** p : {&h->r32b, &h->s32b, &h->w32a, &h->w32b})
            if ((rc = dmalloc(h, p, (size_t)h->ntot))) return rc;
        PCG_CK(h, cudaFuncSetAttribute(pcg::k_sweep_sr<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float) * pcg::SrTile<float>::NH * pcg::SR_MAX_NZ)));
    } else {
        if (h->w64b) return PCG_OK;
        for (double** p : {&h->r64b, &h->s64b, &h->w64a, &h->w64b})
            if ((rc = dmalloc(h, p, (size_t)h->ntot))) return rc;
        PCG_CK(h, cudaFuncSetAttribute(pcg::k_sweep_sr<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(double) * pcg::SrTile<double>::NH * pcg::SR_MAX_NZ)));
    }
    return PCG_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependency on libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    // initialised once, safely when several host threads create handles at once
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000)f;
        return nullptr;
    }();
    return fn;
}

// Tensor map of an FP32 array [nlev][ny][nx] with box bx x by x bz (rows of
// a multiple of 16 bytes: nx % 4 == 0).
bool encode_map_dims(CUtensorMap* m, float* base, long long nx, long long ny, long long nlev, unsigned bx,
                     unsigned by, unsigned bz) {
    auto enc = tensor_map_encoder();
    if (!enc || nx % 4 != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nlev};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)(nx * ny) * 4};
    const cuuint32_t box[3] = {bx, by, bz};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ... of a handle's FP32 vector [nrhs * n_z][n_y][n_x]
bool encode_map(pcg_t h, CUtensorMap* m, float* base, unsigned bx, unsigned by, unsigned bz) {
    return encode_map_dims(m, base, h->nx, h->ny, (long long)h->nz * h->nrhs, bx, by, bz);
}

constexpr int TMA_LZ = 16, TMA_BY = 8;
using SpmvTile = pcg::SpmvTmaTile<TMA_LZ, TMA_BY>;
// persistent pipelined SpMV sweep: 16-level chunks of 32 x 4-column tiles,
// two threads per column (8 levels each)
constexpr int TMA2_LZ = 16, TMA2_BY = 4, TMA2_S = 2;
size_t spmv2_smem(int nz) { return pcg::spmv_tma2_smem<TMA2_LZ, TMA2_BY>(nz); }

int ensure_ws32(pcg_t h) {
    if (h->u32) return PCG_OK;
    int rc;
    for (float** p : {&h->u32, &h->r32, &h->z32, &h->p32, &h->q32})
        if ((rc = dmalloc(h, p, (size_t)h->ntot))) return rc;
    if (h->spmv32 == 4) {
        const unsigned zx = BX + 2 * pcg::TMA_HALO_X;
        const size_t smem = spmv2_smem(h->nz);
        int occ = 0, dev = 0, sms = 1;
        cudaError_t ea = cudaFuncSetAttribute(pcg::k_sweep_spmv_tma2<TMA2_LZ, TMA2_BY, TMA2_S>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ea == cudaSuccess)
            ea = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg::k_sweep_spmv_tma2<TMA2_LZ, TMA2_BY, TMA2_S>,
                                                               BX * TMA2_BY * TMA2_S, smem);
        if (ea == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        h->spmv2_nch = (h->nz + TMA2_LZ - 1) / TMA2_LZ;
        h->spmv2_gx = (h->nx + BX - 1) / BX;
        h->spmv2_gy = (h->ny + TMA2_BY - 1) / TMA2_BY;
        const long long nitems = (long long)h->spmv2_gx * h->spmv2_gy * h->spmv2_nch;
        h->spmv2_G = (int)std::max(1LL, std::min(nitems, (long long)sms * std::max(occ, 1)));
        h->tma2_ready = ea == cudaSuccess && occ >= 1 && nitems < (1LL << 31) &&
                        encode_map(h, &h->tm2_u, h->u32, BX, TMA2_BY, TMA2_LZ) &&
                        encode_map(h, &h->tm2_p, h->p32, BX, TMA2_BY, TMA2_LZ) &&
                        encode_map(h, &h->tm2_q, h->q32, BX, TMA2_BY, TMA2_LZ) &&
                        encode_map(h, &h->tm2_z, h->z32, zx, TMA2_BY + 2, TMA2_LZ + 2);
        if (!h->tma2_ready) {
            cudaGetLastError();
            h->spmv32 = 3;      // the single-stage TMA sweep
        }
    }
    if (h->spmv32 == 3) {
        // the TMA SpMV sweep: maps of the workspace vectors; fall back to the
        // chunked sweep when the driver cannot encode them
        const unsigned zx = BX + 2 * pcg::TMA_HALO_X;
        const unsigned by = (unsigned)h->tma_by;
        h->tma_ready = encode_map(h, &h->tm_u, h->u32, BX, by, TMA_LZ) &&
                       encode_map(h, &h->tm_p, h->p32, BX, by, TMA_LZ) &&
                       encode_map(h, &h->tm_q, h->q32, BX, by, TMA_LZ) &&
                       encode_map(h, &h->tm_z, h->z32, zx, by + 2, TMA_LZ + 2) &&
                       (h->tma_by == 4
                            ? cudaFuncSetAttribute(pcg::k_sweep_spmv_tma<TMA_LZ, 4>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)pcg::SpmvTmaTile<TMA_LZ, 4>::SMEM)
                            : cudaFuncSetAttribute(pcg::k_sweep_spmv_tma<TMA_LZ, TMA_BY>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)SpmvTile::SMEM)) == cudaSuccess;
        if (!h->tma_ready) h->spmv32 = (h->chunked32 && h->plane * (long long)h->nrhs < (1LL << 19)) ? 1 : 0;
    }
    if (h->prec32 == 2) {
        const unsigned lev = (unsigned)(((h->nz + h->lz_a - 1) / h->lz_a) * h->lz_a);
        int occ = 0;
        cudaError_t ea = cudaSuccess;
        for (auto fn : {pcg::k_sweep_prec_tma<16, 0>, pcg::k_sweep_prec_tma<16, 1>, pcg::k_sweep_prec_tma<16, 2>,
                        pcg::k_sweep_prec_tma<16, 4>, pcg::k_sweep_prec_tma<16, 8>})
            if (ea == cudaSuccess)
                ea = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pcg::PrecTmaTile<16>::SMEM);
        if (ea == cudaSuccess)
            ea = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg::k_sweep_prec_tma<16, 1>, 256,
                                                               pcg::PrecTmaTile<16>::SMEM);
        int dev = 0, sms = 1;
        if (ea == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        h->prec_tma_ready = ea == cudaSuccess && occ >= 1 &&
                            encode_map(h, &h->tm_pr, h->r32, BX, (unsigned)h->prec_R, lev) &&
                            encode_map(h, &h->tm_pq, h->q32, BX, (unsigned)h->prec_R, lev);
        // persistent grid per right-hand side: the resident blocks of every SM.
        // It does not depend on nrhs, so that each right-hand side's sums are
        // formed in the same order alone and in a batch.
        h->prec_G = std::max(1, std::min(h->prec_items, sms * std::max(occ, 1)));
        if (!h->prec_tma_ready) h->prec32 = 0;
    }
    return PCG_OK;
}

// Launch a kernel, with programmatic stream serialization when pdl is set
// (the kernel then overlaps the end of the previous one in the stream up to
// its pdl_wait(); only kernels that call it may be launched this way).
template <typename... KArgs, typename... Args>
void launch_pdl(bool pdl, void (*kern)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s, Args... args) {
    if (!pdl) {
        kern<<<g, b, smem, s>>>(args...);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, args...);
}

// Launch the preconditioner sweep / SpMV sweep in the variant chosen at creation.
template <typename T>
bool use_chunked(pcg_t h) { return sizeof(T) == 4 ? h->chunked32 != 0 : h->chunked64 != 0; }

template <typename T>
void launch_prec(pcg_t h, cudaStream_t s, const OpView<T>& v, T* r, T* q, T* z, SolveState* st, bool pdl = false) {
    const bool chunked = use_chunked<T>(h);
    if constexpr (sizeof(T) == 4) {
        if (h->prec32 == 2 && h->prec_tma_ready && r == h->r32 && q == h->q32 && z == h->z32) {
            const dim3 grid(h->prec_G, h->nrhs, 1), block(BX, 8, 1);
            const int nch = (h->nz + h->lz_a - 1) / h->lz_a;
            // one factor set for all columns: per-level carry tables (bitwise the same solve)
#define PCG_PREC_TMA(RT)                                                                                     \
    launch_pdl(pdl, pcg::k_sweep_prec_tma<16, RT>, grid, block, pcg::PrecTmaTile<16>::SMEM, s, v, h->tm_pr,      \
               h->tm_pq, r, (const T*)q, z, st, h->partials, h->counters, h->prec_R, nch, h->prec_gx, h->prec_items)
            if (h->cls_mode != 0 || h->prec_generic) PCG_PREC_TMA(0);
            else if (h->prec_R == 1) PCG_PREC_TMA(1);
            else if (h->prec_R == 2) PCG_PREC_TMA(2);
            else if (h->prec_R == 4) PCG_PREC_TMA(4);
            else PCG_PREC_TMA(8);
#undef PCG_PREC_TMA
            return;
        }
    }
#define PCG_PREC_CH(LZ, MB)                                                                                  \
    pcg::k_sweep_prec_chunked<T, LZ, MB><<<h->grid_a, h->block_a, 0, s>>>(v, r, q, z, st, h->partials, h->counters, \
                                                                          h->nblk_a)
    if (chunked && h->lz_a == 16) {
        // three resident blocks asked of the compiler (85-register cap, no
        // spills): 9-13 % faster than the uncapped 108 registers at 256^2,
        // 1024^2 and the shell
        PCG_PREC_CH(16, 3);
    } else if (chunked) {
        PCG_PREC_CH(32, 1);
    } else {
        // loads issued ahead while the grid has few columns (65536 columns:
        // 155 -> 113 us per sweep); plain loop beyond (2^20 columns: 1505 vs
        // 1634 us, where the extra registers cost more occupancy than they gain)
        if (sizeof(T) == 8 && h->plane * (long long)h->nrhs < (1LL << 19))
            pcg::k_sweep_prec<T, true><<<h->grid_c, h->block_c, 0, s>>>(v, r, q, z, st, h->partials, h->counters,
                                                                         h->nblk_c);
        else
            pcg::k_sweep_prec<T, false><<<h->grid_c, h->block_c, 0, s>>>(v, r, q, z, st, h->partials, h->counters,
                                                                          h->nblk_c);
    }
#undef PCG_PREC_CH
}

template <typename T>
void launch_spmv(pcg_t h, cudaStream_t s, const OpView<T>& v, T* u, T* p, T* q, T* z, SolveState* st,
                 bool pdl = false) {
    const int mode = sizeof(T) == 4 ? h->spmv32 : h->spmv64;
#define PCG_SPMV_CH(LZ, MB)                                                                                  \
    pcg::k_sweep_spmv_chunked<T, LZ, MB><<<h->grid_b, h->block_b, 0, s>>>(v, u, p, q, z, st, h->partials,      \
                                                                          h->counters, h->nblk_b, h->nch_b)
    if constexpr (sizeof(T) == 4) {
        if (mode == 4 && h->tma2_ready && u == h->u32 && p == h->p32 && q == h->q32 && z == h->z32) {
            launch_pdl(pdl, pcg::k_sweep_spmv_tma2<TMA2_LZ, TMA2_BY, TMA2_S>, dim3(h->spmv2_G, h->nrhs, 1),
                       dim3(BX, TMA2_BY * TMA2_S, 1), spmv2_smem(h->nz), s, v, h->tm2_u, h->tm2_p, h->tm2_q, h->tm2_z, u, p, q,
                       (const T*)z, st, h->partials, h->counters, h->spmv2_gx, h->spmv2_gy, h->spmv2_nch);
            return;
        }
        if (mode == 3 && h->tma_ready && u == h->u32 && p == h->p32 && q == h->q32 && z == h->z32) {
            if (h->tma_by == 4)
                pcg::k_sweep_spmv_tma<TMA_LZ, 4><<<h->grid_t, h->block_t, pcg::SpmvTmaTile<TMA_LZ, 4>::SMEM, s>>>(
                    v, h->tm_u, h->tm_p, h->tm_q, h->tm_z, u, p, q, z, st, h->partials, h->counters, h->nblk_t,
                    h->nch_b);
            else
                pcg::k_sweep_spmv_tma<TMA_LZ, TMA_BY><<<h->grid_t, h->block_t, SpmvTile::SMEM, s>>>(
                    v, h->tm_u, h->tm_p, h->tm_q, h->tm_z, u, p, q, z, st, h->partials, h->counters, h->nblk_t,
                    h->nch_b);
            return;
        }
    }
    if (mode == 1 || mode >= 3) {
        PCG_SPMV_CH(16, 1);
    } else {
        const dim3 g(h->grid_c.x, h->grid_c.y, h->grid_c.z * h->ksplit);
        if (sizeof(T) == 8 && h->spmv_pipe)
            pcg::k_sweep_spmv<T, true><<<g, h->block_c, 0, s>>>(v, u, p, q, z, st, h->partials, h->counters,
                                                                h->nblk_c * h->ksplit, h->ksplit);
        else
            pcg::k_sweep_spmv<T, false><<<g, h->block_c, 0, s>>>(v, u, p, q, z, st, h->partials, h->counters,
                                                                 h->nblk_c * h->ksplit, h->ksplit);
    }
#undef PCG_SPMV_CH
}

// One V-cycle z0 = B r0 (PCG_PREC_MULTIGRID) on stream s, in precision V:
// level 0 is the handle itself (scratch t0), levels 1.. are h->mg.  Returns
// the number of kernels launched.  st: per-rhs states (a stopped rhs is
// skipped).
template <typename V>
OpView<V> level_view(pcg_t hl) {
    if constexpr (sizeof(V) == 8) return hl->view64();
    else return hl->view32();
}

// Launch shapes of the multigrid's elementwise kernels (x: cells of one
// right-hand side, y: right-hand sides) and of its transfers (x: tiles of a
// level, y: levels, z: right-hand sides).
dim3 elem_grid(long long vol, int nrhs) {
    return dim3((unsigned)std::min<long long>((vol + 255) / 256, 152LL * 16), (unsigned)std::min(nrhs, 65535));
}

struct CellLaunch {
    dim3 g, b;
    int nbi;
};

CellLaunch cell_launch(int nx, int ny, int nz, int nrhs) {
    const int bx = nx >= 128 ? 128 : (nx >= 64 ? 64 : 32), by = 256 / bx;
    const int nbi = (nx + bx - 1) / bx;
    const long long gx = (long long)nbi * ((ny + by - 1) / by);
    const int gy = std::min((nz + 3) / 4, 65535);     // four levels per thread
    return {dim3((unsigned)gx, (unsigned)gy, (unsigned)std::min(nrhs, 65535)), dim3(bx, by), nbi};
}

template <typename V>
int launch_vcycle(pcg_t h, cudaStream_t s, const SolveState* st, const V* r0, V* z0, V* t0) {
    const int L = (int)h->mg.size() + 1;
    auto H = [&](int l) { return l == 0 ? h : h->mg[l - 1].h; };
    auto lv = [&](int l, double* d, float* f) -> V* {
        (void)d; (void)f;
        if constexpr (sizeof(V) == 8) return d; else return f;
    };
    auto R = [&](int l) -> const V* { return l == 0 ? r0 : lv(l, h->mg[l - 1].r, h->mg[l - 1].rf); };
    auto Z = [&](int l) -> V* { return l == 0 ? z0 : lv(l, h->mg[l - 1].z, h->mg[l - 1].zf); };
    auto T = [&](int l) -> V* { return l == 0 ? t0 : lv(l, h->mg[l - 1].t, h->mg[l - 1].tf); };
    const V omega = (V)h->mg_omega;
    int n = 0;
    // Each column's work is spread over several threads where a level has too
    // few columns to keep the SMs' loads in flight: the residual over level
    // chunks (parts of a column), and the line solve in its chunked form (one
    // warp per 16 levels) with the damped update as its store.  In FP32 the
    // chunked form is the faster one on every level (it keeps more loads in
    // flight and has no y round trip through memory); in FP64, bound by the
    // FP64 pipe, its extra arithmetic makes it slower on large levels.
    const long long few_cols = sizeof(V) == 4 ? std::numeric_limits<long long>::max() : 16384;
    auto few = [&](pcg_t hl) { return hl->plane * (long long)hl->nrhs < few_cols && hl->nz <= 128; };
    auto ksplit = [&](pcg_t hl) {
        int ks = 1;
        while (hl->plane * (long long)hl->nrhs * ks < h->mg_resid_threads && ks < 32 && hl->nz / (2 * ks) >= 4 &&
               (long long)hl->nrhs * ks * 2 <= 65535)
            ks *= 2;
        return ks;
    };
    // FP32 levels whose rows split into quads, whose row count is even and
    // that have at least mg_quad columns take the residual kernels on float4
    // quads of row pairs (k_mg_resid4): fewer loads and instructions per cell
    // where the level is large enough to be bound by them; on smaller levels
    // the scalar kernels' thread per column keeps more loads in flight.
    auto quad = [&](pcg_t hl) {
        return sizeof(V) == 4 && h->mg_quad > 0 && hl->plane >= h->mg_quad && hl->nx % 4 == 0 && hl->ny % 2 == 0;
    };
    auto resid4 = [&](int l, int mode, V* out) {
        if constexpr (sizeof(V) == 4) {
            pcg_t hl = H(l);
            const long long units = (long long)(hl->ny / 2) * (hl->nx / 4);
            int ks = 1;
            // one thread per eight cells: half the scalar kernels' thread target
            while (units * hl->nrhs * ks < h->mg_resid_threads / 2 && ks < 32 && hl->nz / (2 * ks) >= 4 &&
                   (long long)hl->nrhs * ks * 2 <= 65535)
                ks *= 2;
            const dim3 g((unsigned)((units + 127) / 128), 1, (unsigned)(hl->nrhs * ks));
            const pcg::OpView<float> v = level_view<V>(hl);
            if (mode == 0)
                pcg::k_mg_resid4<0><<<g, 128, 0, s>>>(v, R(l), Z(l), out, st, ks);
            else
                pcg::k_mg_resid4<1><<<g, 128, 0, s>>>(v, R(l), Z(l), out, st, ks);
            ++n;
        }
    };
    auto resid = [&](int l) {                            // t = r - A z
        pcg_t hl = H(l);
        if (quad(hl)) {
            resid4(l, 0, T(l));
            return;
        }
        const int ks = ksplit(hl);
        const dim3 g(hl->grid_c.x, hl->grid_c.y, hl->grid_c.z * ks);
        // the loads of the next 4 (FP32) or 2 (FP64) levels in flight
        if constexpr (sizeof(V) == 4)
            pcg::k_mg_resid<V, 4><<<g, hl->block_c, 0, s>>>(level_view<V>(hl), R(l), Z(l), T(l), st, ks);
        else
            pcg::k_mg_resid<V, 2><<<g, hl->block_c, 0, s>>>(level_view<V>(hl), R(l), Z(l), T(l), st, ks);
        ++n;
    };
    auto smooth = [&](int l, const V* rin, V om, int acc) {   // z = (acc ? z : 0) + omega M^{-1} rin
        pcg_t hl = H(l);
        if (few(hl)) {
            const int nch = (hl->nz + 15) / 16;
            pcg::k_mg_lsolve_chunked<V><<<dim3((hl->nx + 31) / 32, hl->ny, hl->nrhs), dim3(32, nch, 1), 0, s>>>(
                level_view<V>(hl), rin, Z(l), om, acc, st);
            ++n;
        } else {
            pcg::k_mg_smooth<V><<<hl->grid_c, hl->block_c, 0, s>>>(level_view<V>(hl), rin, T(l), Z(l), om, acc, st);
            ++n;
        }
    };
    auto smooth_first = [&](int l, V om) { smooth(l, R(l), om, 0); };   // z = omega M^{-1} r
    auto smooth_more = [&](int l) {                      // z += omega M^{-1} (r - A z)
        resid(l);
        smooth(l, T(l), omega, 1);
    };
    // Levels lt .. L-1 (at most mg_tail_cols columns each, all solved in the
    // chunked form, their r and z and one residual scratch within
    // mg_tail_smem bytes) run in one k_mg_tail launch; lt = L: none.
    int lt = L;
    if (h->mg_tail_cols > 0 && h->nrhs <= 65535)
        for (int l = L - 1; l >= 0 && L - l <= pcg::TAIL_MAXL; --l) {
            pcg_t hl = H(l);
            if (hl->plane > h->mg_tail_cols || !few(hl)) break;
            long long elems = 0;
            for (int m = l; m < L; ++m) elems += 2 * ((H(m)->vol + 3) / 4 * 4);
            elems += (hl->vol + 3) / 4 * 4;
            if (elems * (long long)sizeof(V) > h->mg_tail_smem) break;
            lt = l;
        }
    for (int l = 0; l + 1 < L && l < lt; ++l) {
        smooth_first(l, omega);
        for (int k = 1; k < h->mg_nu; ++k) smooth_more(l);
        pcg_t hl = H(l), hc = H(l + 1);
        if (quad(hl)) {                                  // the residual restricted as it is formed
            resid4(l, 1, const_cast<V*>(R(l + 1)));
            continue;
        }
        if (hl->ny / 2 <= 65535) {
            // the residual restricted as it is formed (t is not written)
            const int ks = ksplit(hl);
            const dim3 g((hl->nx + 31) / 32, hl->ny / 2, hl->nrhs * ks);
            if constexpr (sizeof(V) == 4)
                pcg::k_mg_resid_restrict<V, 4><<<g, dim3(32, 2), 0, s>>>(level_view<V>(hl), R(l), Z(l),
                                                                        const_cast<V*>(R(l + 1)), st, ks);
            else
                pcg::k_mg_resid_restrict<V, 2><<<g, dim3(32, 2), 0, s>>>(level_view<V>(hl), R(l), Z(l),
                                                                        const_cast<V*>(R(l + 1)), st, ks);
            ++n;
            continue;
        }
        resid(l);
        const CellLaunch cl = cell_launch(hc->nx, hc->ny, hc->nz, hc->nrhs);
        pcg::k_mg_restrict<V><<<cl.g, cl.b, 0, s>>>(T(l), const_cast<V*>(R(l + 1)), hc->nx, hc->ny, hc->nz, hc->nrhs,
                                                    cl.nbi, st);
        ++n;
    }
    const int c = L - 1;
    if (lt < L) {
        pcg::TailArgs<V> a{};
        a.nlev = L - lt;
        a.nu = h->mg_nu;
        a.ncoarse = h->mg_coarse;
        a.omega = omega;
        a.r_in = R(lt);
        a.z_out = Z(lt);
        long long off = 0;
        for (int l = lt; l < L; ++l) {
            a.op[l - lt] = level_view<V>(H(l));
            a.off_r[l - lt] = off;
            off += (H(l)->vol + 3) / 4 * 4;
            a.off_z[l - lt] = off;
            off += (H(l)->vol + 3) / 4 * 4;
        }
        a.off_t = off;
        off += (H(lt)->vol + 3) / 4 * 4;
        pcg::k_mg_tail<V><<<dim3((unsigned)h->nrhs), dim3(32, pcg::TAIL_WARPS), (size_t)off * sizeof(V), s>>>(a, st);
        ++n;
    } else if (H(c)->plane == 1) {
        // one column: its block is all of A, solved with one step of
        // refinement (z += M^{-1} (r - A z)): without horizontal couplings the
        // block's condition number reaches 1e10 at strong anisotropy
        smooth_first(c, V(1));
        resid(c);
        smooth(c, T(c), V(1), 1);
    } else {
        smooth_first(c, omega);
        for (int k = 1; k < h->mg_coarse; ++k) smooth_more(c);
    }
    for (int l = std::min(L - 2, lt - 1); l >= 0; --l) {
        pcg_t hl = H(l);
        if constexpr (sizeof(V) == 4) {
            if (quad(hl)) {
                const long long units = (long long)hl->ny * (hl->nx / 4);
                const dim3 g((unsigned)((units + 255) / 256), (unsigned)std::min((hl->nz + 3) / 4, 65535),
                             (unsigned)std::min(hl->nrhs, 65535));
                pcg::k_mg_prolong4<<<g, 256, 0, s>>>(Z(l + 1), Z(l), hl->nx, hl->ny, hl->nz, hl->nrhs, st);
                ++n;
                for (int k = 0; k < h->mg_nu; ++k) smooth_more(l);
                continue;
            }
        }
        const CellLaunch cl = cell_launch(hl->nx, hl->ny, hl->nz, hl->nrhs);
        pcg::k_mg_prolong<V><<<cl.g, cl.b, 0, s>>>(Z(l + 1), Z(l), hl->nx, hl->ny, hl->nz, hl->nrhs, cl.nbi, st);
        ++n;
        for (int k = 0; k < h->mg_nu; ++k) smooth_more(l);
    }
    return n;
}

// Opt k_mg_tail in to the shared memory its levels need (the block's
// static arrays come on top); on failure the coarse levels run as separate
// launches.
template <typename V>
bool tail_smem_ok(pcg_t h) {
    if (cudaFuncSetAttribute(pcg::k_mg_tail<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->mg_tail_smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

bool tail_ready(pcg_t h) { return h->mg_f32 ? tail_smem_ok<float>(h) : tail_smem_ok<double>(h); }

// Levels of the multigrid hierarchy: n_x, n_y halved while both are even
// (down to one column), each level a handle of its own on the coarser grid
// with alpha on a coarse face the mean of its two fine faces.
int build_hierarchy(pcg_t h, const pcg_grid_t* grid, const pcg_coeffs_t* coeffs) {
    int rc;
    if ((rc = dmalloc(h, &h->mg_t0, (size_t)h->ntot))) return rc;
    if (h->mg_f32)
        for (float** p : {&h->mg_r0f, &h->mg_z0f, &h->mg_t0f})
            if ((rc = dmalloc(h, p, (size_t)h->ntot))) return rc;
    if ((rc = dmalloc(h, &h->mg_free, h->nrhs))) return rc;
    PCG_CK(h, cudaMemsetAsync(h->mg_free, 0, sizeof(SolveState) * h->nrhs, h->stream));
    pcg_grid_t g = *grid;
    std::vector<double> ae, an;
    if (coeffs->alpha_e) ae.assign(coeffs->alpha_e, coeffs->alpha_e + (size_t)g.n_x * g.n_y);
    if (coeffs->alpha_n) an.assign(coeffs->alpha_n, coeffs->alpha_n + (size_t)g.n_x * g.n_y);
    while (h->mg.size() < 31 && g.n_x % 2 == 0 && g.n_y % 2 == 0 && (long long)g.n_x * g.n_y > 1) {
        const int nx = g.n_x, nxc = g.n_x / 2, nyc = g.n_y / 2;
        std::vector<double> aec, anc;
        if (!ae.empty()) {
            aec.resize((size_t)nxc * nyc);
            for (int J = 0; J < nyc; ++J)
                for (int I = 0; I < nxc; ++I)
                    aec[(size_t)J * nxc + I] = 0.5 * (ae[(size_t)(2 * J) * nx + 2 * I + 1] + ae[(size_t)(2 * J + 1) * nx + 2 * I + 1]);
        }
        if (!an.empty()) {
            anc.resize((size_t)nxc * nyc);
            for (int J = 0; J < nyc; ++J)
                for (int I = 0; I < nxc; ++I)
                    anc[(size_t)J * nxc + I] = 0.5 * (an[(size_t)(2 * J + 1) * nx + 2 * I] + an[(size_t)(2 * J + 1) * nx + 2 * I + 1]);
        }
        g.n_x = nxc;
        g.n_y = nyc;
        pcg_coeffs_t c = *coeffs;
        c.alpha_e = aec.empty() ? nullptr : aec.data();
        c.alpha_n = anc.empty() ? nullptr : anc.data();
        pcg_opts_t o{};
        o.precision = PCG_FP64;
        o.passes_per_launch = h->ppl;
        o.stream = (void*)h->stream;
        o.preconditioner = PCG_PREC_LINE;
        pcg_t hc = nullptr;
        rc = pcg_create(&g, &c, &o, &hc);
        if (rc) return fail(h, rc, "multigrid level " + std::to_string(h->mg.size() + 1) + ": " + g_create_error);
        h->mg.push_back(pcg_ctx::MGLevel{});
        h->mg.back().h = hc;
        if (h->mg_f32) {
            for (float** p : {&h->mg.back().rf, &h->mg.back().zf, &h->mg.back().tf})
                if ((rc = dmalloc(h, p, (size_t)hc->ntot))) return rc;
        } else {
            for (double** p : {&h->mg.back().r, &h->mg.back().z, &h->mg.back().t})
                if ((rc = dmalloc(h, p, (size_t)hc->ntot))) return rc;
        }
        ae.swap(aec);
        an.swap(anc);
    }
    return PCG_OK;
}

// One Algorithm-1 pass with the V-cycle as preconditioner: r <- r - alpha q;
// z = B r; <r, r>, <r, z>, stopping test, beta; then the SpMV sweep.
int launch_mg_pass(pcg_t h, cudaStream_t s) {
    const dim3 g = elem_grid(h->vol, h->nrhs);
    // an FP32 cycle takes r rounded as it is updated, and its z is widened
    // as the dot products read it
    pcg::k_mg_rupdate<<<g, 256, 0, s>>>(h->r64, h->q64, h->mg_f32 ? h->mg_r0f : nullptr, h->vol, h->nrhs, h->st);
    int n = 1;
    if (h->mg_f32)
        n += launch_vcycle<float>(h, s, h->st, h->mg_r0f, h->mg_z0f, h->mg_t0f);
    else
        n += launch_vcycle<double>(h, s, h->st, h->r64, h->z64, h->mg_t0);
    pcg::k_mg_dots<<<h->grid_c, h->block_c, 0, s>>>(h->view64(), h->r64, h->z64, h->mg_f32 ? h->mg_z0f : nullptr,
                                                    h->st, h->partials, h->counters, h->nblk_c);
    launch_spmv<double>(h, s, h->view64(), h->u64, h->p64, h->q64, h->z64, h->st);
    return n + 2;
}

// Capture `ppl` passes of Algorithm 1 (preconditioner sweep + SpMV sweep).
template <typename T>
int capture_passes(pcg_t h, OpView<T> v, T* u, T* r, T* z, T* p, T* q, SolveState* st, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    PCG_CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < h->ppl; ++i) {
        if constexpr (sizeof(T) == 8) {
            if (h->precond == PCG_PREC_MULTIGRID) {
                h->kernels_per_pass = launch_mg_pass(h, h->cap_stream);
                continue;
            }
        }
        launch_prec<T>(h, h->cap_stream, v, r, q, z, st, h->pdl != 0);
        launch_spmv<T>(h, h->cap_stream, v, u, p, q, z, st, h->pdl != 0);
    }
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess) return fail(h, PCG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, PCG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return PCG_OK;
}

// Capture `ppl` passes of the single-reduction PCG (one k_sweep_sr each);
// pass i reads buffer i % 2 of r, s, w and writes the other one.
template <typename T>
int capture_passes_sr(pcg_t h, OpView<T> v, T* x, T* u, T* p, T* ra, T* rb, T* sa, T* sb, T* wa, T* wb,
                      SolveState* st, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    const size_t smem = sizeof(T) * pcg::SrTile<T>::NH * h->nz;
    T* rr[2] = {ra, rb};
    T* ss[2] = {sa, sb};
    T* ww[2] = {wa, wb};
    PCG_CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < h->ppl; ++i) {
        const int a = i & 1, b = a ^ 1;
        pcg::k_sweep_sr<T><<<h->grid_sr, pcg::SrTile<T>::NT, smem, h->cap_stream>>>(
            v, x, u, p, rr[a], rr[b], ss[a], ss[b], ww[a], ww[b], st, h->partials, h->counters, h->nblk_sr);
    }
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess) return fail(h, PCG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, PCG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    h->kernels_per_pass = 1;
    return PCG_OK;
}

// Run passes until every rhs is done (or `max_launch` graph launches).
// Two graph launches are kept in flight; after each, the per-rhs states are
// copied to a pinned slot and polled when the launch's event completes.
int run_graph(pcg_t h, cudaGraphExec_t graph, SolveState* st, long long max_launch) {
    const size_t sb = sizeof(SolveState) * h->nrhs;
    long long issued = 0, polled = 0;
    bool all_done = false;
    auto issue = [&](long long n) -> int {
        PCG_CK(h, cudaGraphLaunch(graph, h->stream));
        PCG_CK(h, cudaMemcpyAsync(h->h_st + (n & 1) * h->nrhs, st, sb, cudaMemcpyDeviceToHost, h->stream));
        PCG_CK(h, cudaEventRecord(h->ev[n & 1], h->stream));
        h->launches += (long long)h->kernels_per_pass * h->ppl;
        return PCG_OK;
    };
    int rc;
    if ((rc = issue(issued++))) return rc;
    while (!all_done && polled < max_launch) {
        if (issued < max_launch && issued == polled + 1)
            if ((rc = issue(issued++))) return rc;
        PCG_CK(h, cudaEventSynchronize(h->ev[polled & 1]));
        const SolveState* s = h->h_st + (polled & 1) * h->nrhs;
        all_done = true;
        for (int r = 0; r < h->nrhs; ++r) all_done = all_done && s[r].done;
        ++polled;
    }
    PCG_CK(h, cudaStreamSynchronize(h->stream));
    return PCG_OK;
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int solve_fp64(pcg_t h, const double* b, double* x, double tol, int maxit, pcg_stats_t* stats) {
    int rc;
    if ((rc = ensure_ws64(h))) return rc;
    if (h->alg_sr) {   // x is u64, u is z64, p is p64, s is q64 / s64b
        if ((rc = ensure_ws_sr(h, false))) return rc;
        if (!h->graph_sr &&
            (rc = capture_passes_sr<double>(h, h->view64(), h->u64, h->z64, h->p64, h->r64, h->r64b, h->q64, h->s64b,
                                            h->w64a, h->w64b, h->st, &h->graph_sr)))
            return rc;
    } else if (!h->graph64) {
        if ((rc = capture_passes<double>(h, h->view64(), h->u64, h->r64, h->z64, h->p64, h->q64, h->st, &h->graph64)))
            return rc;
    }
    const OpView<double> v = h->view64();
    cudaStream_t s = h->stream;
    h->launches = 0;
    pcg::k_init_state<<<(h->nrhs + 63) / 64, 64, 0, s>>>(h->st, h->nrhs, tol * tol, maxit, nullptr);
    pcg::k_residual<double><<<h->grid, h->block, 0, s>>>(v, b, x, h->u64, h->r64, h->st, h->partials, h->counters,
                                                        h->nblocks, 0);
    PCG_CK(h, cudaMemsetAsync(h->p64, 0, sizeof(double) * h->ntot, s));
    PCG_CK(h, cudaMemsetAsync(h->q64, 0, sizeof(double) * h->ntot, s));
    if (h->alg_sr) {   // u = w = 0 before the first pass (p and s are cleared above)
        PCG_CK(h, cudaMemsetAsync(h->z64, 0, sizeof(double) * h->ntot, s));
        PCG_CK(h, cudaMemsetAsync(h->w64a, 0, sizeof(double) * h->ntot, s));
    }
    PCG_CK(h, cudaGetLastError());
    h->launches += 2;
    const long long max_launch = ((long long)maxit + 1 + h->ppl - 1) / h->ppl + 1;
    if ((rc = run_graph(h, h->alg_sr ? h->graph_sr : h->graph64, h->st, max_launch))) return rc;
    pcg::k_finish<<<h->grid, h->block, 0, s>>>(h->nx, h->ny, h->nz, h->plane, h->vol, x, h->u64, h->p64, h->st);
    pcg::k_residual<double><<<h->grid, h->block, 0, s>>>(v, b, x, nullptr, (double*)nullptr, h->st, h->partials,
                                                        h->counters, h->nblocks, 1);
    PCG_CK(h, cudaGetLastError());
    h->launches += 2;
    PCG_CK(h, cudaMemcpyAsync(h->h_st, h->st, sizeof(SolveState) * h->nrhs, cudaMemcpyDeviceToHost, s));
    PCG_CK(h, cudaStreamSynchronize(s));
    int worst = PCG_OK;
    for (int r = 0; r < h->nrhs; ++r) {
        const SolveState& q = h->h_st[r];
        pcg_stats_t& o = h->rhs_stats[r];
        o = pcg_stats_t{};
        o.status = q.done ? q.status : PCG_NOT_CONVERGED;
        o.iterations = std::max(0, q.pass - 1);
        o.outer_sweeps = 0;
        o.relres_recursive = q.bnorm2 > 0 ? std::sqrt(q.rr / q.bnorm2) : 0.0;
        o.relres_true = q.bnorm2 > 0 ? std::sqrt(q.rr_true / q.bnorm2) : 0.0;
        o.relres_floor = q.bnorm2 > 0 ? std::sqrt(q.floor2 / q.bnorm2) : 0.0;
        if (o.status != PCG_OK && worst == PCG_OK) worst = o.status;
        if (o.status == PCG_BREAKDOWN) worst = PCG_BREAKDOWN;
    }
    (void)stats;
    return worst;
}

int solve_mixed(pcg_t h, const double* b, double* x, double tol, int maxit, pcg_stats_t* stats) {
    int rc;
    if ((rc = ensure_ws32(h))) return rc;
    if (h->alg_sr) {   // inner solve: e is u32, u is z32, p is p32, s is q32 / s32b
        if ((rc = ensure_ws_sr(h, true))) return rc;
        if (!h->graph_sr32 &&
            (rc = capture_passes_sr<float>(h, h->view32(), h->u32, h->z32, h->p32, h->r32, h->r32b, h->q32, h->s32b,
                                           h->w32a, h->w32b, h->st_in, &h->graph_sr32)))
            return rc;
    } else if (!h->graph32) {
        if ((rc = capture_passes<float>(h, h->view32(), h->u32, h->r32, h->z32, h->p32, h->q32, h->st_in, &h->graph32)))
            return rc;
    }
    const int inner_cap = (maxit > 0 && maxit < h->inner_maxit) ? maxit : h->inner_maxit;
    const OpView<double> v = h->view64();
    cudaStream_t s = h->stream;
    const int nr = h->nrhs;
    h->launches = 0;
    std::vector<int> active(nr, 1), done(nr, 0), status(nr, PCG_NOT_CONVERGED), stag(nr, 0), sweeps(nr, 0), inner_it(nr, 0);
    std::vector<std::vector<double>> hist(nr);
    std::vector<double> bb(nr, 0.0), last_rr(nr, 0.0), floor_rel(nr, 0.0);
    pcg::k_init_state<<<(nr + 63) / 64, 64, 0, s>>>(h->st, nr, tol * tol, 0, nullptr);
    h->launches += 1;
    for (int m = 0; m <= h->max_outer; ++m) {
        // true residual of x in FP64 (its norm decides; its sum gives the coarse correction)
        pcg::k_residual<float><<<h->grid, h->block, 0, s>>>(v, b, x, nullptr, (float*)nullptr, h->st, h->partials,
                                                           h->counters, h->nblocks, 2);
        PCG_CK(h, cudaGetLastError());
        h->launches += 1;
        PCG_CK(h, cudaMemcpyAsync(h->h_st, h->st, sizeof(SolveState) * nr, cudaMemcpyDeviceToHost, s));
        PCG_CK(h, cudaStreamSynchronize(s));
        bool any = false;
        for (int r = 0; r < nr; ++r) {
            active[r] = 0;
            if (done[r]) continue;
            const double rrv = h->h_st[r].rr;
            bb[r] = h->h_st[r].bnorm2;
            last_rr[r] = rrv;
            if (bb[r] == 0.0) {     // the solution is zero
                PCG_CK(h, cudaMemsetAsync(x + (size_t)r * h->vol, 0, sizeof(double) * h->vol, s));
                done[r] = 1;
                status[r] = PCG_OK;
                last_rr[r] = 0.0;
                continue;
            }
            const double rel = std::sqrt(rrv / bb[r]);
            floor_rel[r] = std::sqrt(h->h_st[r].floor2 / bb[r]);
            hist[r].push_back(rel);
            if (h->trace) std::fprintf(stderr, "[pcg] rhs %d sweep %d relres_true %.3e floor %.3e inner_its_so_far %d\n", r, m, rel, floor_rel[r], inner_it[r]);
            if (!std::isfinite(rel)) { done[r] = 1; status[r] = PCG_BREAKDOWN; continue; }
            if (rel < tol) { done[r] = 1; status[r] = PCG_OK; continue; }
            // within twice the residual of x rounded to FP64: no FP64 vector does better
            if (rel <= 2.0 * floor_rel[r]) { done[r] = 1; status[r] = PCG_OK; stag[r] = 1; continue; }
            const size_t n = hist[r].size();
            if (n >= 4) {
                // backstop for true stagnation (the floor test above ends normal solves):
                // the best residual has not halved over the last three sweeps
                const double best_now = *std::min_element(hist[r].begin(), hist[r].end());
                const double best_before = *std::min_element(hist[r].begin(), hist[r].end() - 3);
                if (best_now > 0.5 * best_before) { done[r] = 1; status[r] = PCG_OK; stag[r] = 1; continue; }
            }
            if (m == h->max_outer) { done[r] = 1; status[r] = PCG_NOT_CONVERGED; continue; }
            active[r] = 1;
            any = true;
        }
        if (!any) break;
        // coarse correction with the constant vector, then the inner right-hand side
        // r' = b - A x - c A 1 in FP32
        pcg::k_coarse<<<(nr + 63) / 64, 64, 0, s>>>(h->st, nr, h->total_mass);
        pcg::k_residual<float><<<h->grid, h->block, 0, s>>>(v, b, x, nullptr, h->r32, h->st, h->partials,
                                                           h->counters, h->nblocks, 3);
        PCG_CK(h, cudaGetLastError());
        h->launches += 2;
        PCG_CK(h, cudaMemcpyAsync(h->d_active, active.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, s));
        pcg::k_init_state<<<(nr + 63) / 64, 64, 0, s>>>(h->st_in, nr, 0.0, inner_cap, h->d_active);
        pcg::k_inner_thresholds<<<(nr + 63) / 64, 64, 0, s>>>(h->st_in, h->st, nr, h->inner_tol * h->inner_tol);
        PCG_CK(h, cudaMemsetAsync(h->u32, 0, sizeof(float) * h->ntot, s));
        PCG_CK(h, cudaMemsetAsync(h->p32, 0, sizeof(float) * h->ntot, s));
        PCG_CK(h, cudaMemsetAsync(h->q32, 0, sizeof(float) * h->ntot, s));
        if (h->alg_sr) {   // u = w = 0 before the first pass
            PCG_CK(h, cudaMemsetAsync(h->z32, 0, sizeof(float) * h->ntot, s));
            PCG_CK(h, cudaMemsetAsync(h->w32a, 0, sizeof(float) * h->ntot, s));
        }
        PCG_CK(h, cudaGetLastError());
        h->launches += 2;
        const long long max_launch = ((long long)inner_cap + 1 + h->ppl - 1) / h->ppl + 1;
        if ((rc = run_graph(h, h->alg_sr ? h->graph_sr32 : h->graph32, h->st_in, max_launch))) return rc;
        pcg::k_refine_update<<<h->grid, h->block, 0, s>>>(h->nx, h->ny, h->nz, h->plane, h->vol, x, h->u32, h->p32,
                                                         h->st_in, h->st, h->d_active);
        PCG_CK(h, cudaGetLastError());
        h->launches += 1;
        PCG_CK(h, cudaMemcpyAsync(h->h_st + nr, h->st_in, sizeof(SolveState) * nr, cudaMemcpyDeviceToHost, s));
        PCG_CK(h, cudaStreamSynchronize(s));
        for (int r = 0; r < nr; ++r) {
            if (!active[r]) continue;
            sweeps[r] += 1;
            inner_it[r] += std::max(0, h->h_st[nr + r].pass - 1);
            const int is = h->h_st[nr + r].status;
            // The single-reduction inner solve stops (alpha = 0, its correction so
            // far kept) when FP32 rounding makes delta - beta gamma / alpha_old
            // non-positive; the FP64 residual of the next sweep decides, and a
            // non-finite one ends the solve there.
            if (is == PCG_TIMEOUT || (is == PCG_BREAKDOWN && !h->alg_sr)) { done[r] = 1; status[r] = is; }
        }
    }
    int worst = PCG_OK;
    for (int r = 0; r < nr; ++r) {
        pcg_stats_t& o = h->rhs_stats[r];
        o = pcg_stats_t{};
        o.status = done[r] ? status[r] : PCG_NOT_CONVERGED;
        o.iterations = inner_it[r];
        o.outer_sweeps = sweeps[r];
        o.stagnated = stag[r];
        o.relres_true = bb[r] > 0 ? std::sqrt(last_rr[r] / bb[r]) : 0.0;
        o.relres_floor = floor_rel[r];
        o.relres_recursive = o.relres_true;
        if (o.status != PCG_OK && worst == PCG_OK) worst = o.status;
        if (o.status == PCG_BREAKDOWN) worst = PCG_BREAKDOWN;
    }
    (void)stats;
    return worst;
}

void summarise(pcg_t h, pcg_stats_t* stats, int rc, double t0) {
    if (!stats) return;
    pcg_stats_t s{};
    s.status = rc;
    for (int r = 0; r < h->nrhs; ++r) {
        const pcg_stats_t& o = h->rhs_stats[r];
        s.iterations = std::max(s.iterations, o.iterations);
        s.outer_sweeps = std::max(s.outer_sweeps, o.outer_sweeps);
        s.stagnated = std::max(s.stagnated, o.stagnated);
        s.relres_recursive = std::max(s.relres_recursive, o.relres_recursive);
        s.relres_true = std::max(s.relres_true, o.relres_true);
        s.relres_floor = std::max(s.relres_floor, o.relres_floor);
    }
    s.elapsed_ms = now_ms() - t0;
    *stats = s;
}

}  // namespace

extern "C" {

int pcg_create(const pcg_grid_t* grid, const pcg_coeffs_t* coeffs, const pcg_opts_t* opts, pcg_t* out) {
    if (!out) return fail(nullptr, PCG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!grid || !coeffs) return fail(nullptr, PCG_ERR_INVALID_ARG, "grid and coeffs are required");
    if (grid->n_x < 1 || grid->n_y < 1 || grid->n_z < 1 || grid->nrhs < 1)
        return fail(nullptr, PCG_ERR_INVALID_ARG, "n_x, n_y, n_z and nrhs must be >= 1");
    if (!grid->z_iface || !coeffs->beta_iface) return fail(nullptr, PCG_ERR_INVALID_ARG, "z_iface and beta_iface are required");
    if (!(coeffs->lambda2 >= 0.0) || !std::isfinite(coeffs->lambda2))
        return fail(nullptr, PCG_ERR_INVALID_ARG, "lambda2 must be finite and >= 0");
    const long long plane = (long long)grid->n_x * grid->n_y;
    if (plane > (1LL << 31) - 1) return fail(nullptr, PCG_ERR_INVALID_ARG, "n_x * n_y too large");
    pcg_ctx* h = new (std::nothrow) pcg_ctx();
    if (!h) return fail(nullptr, PCG_ERR_OOM, "host allocation failed");
    h->geometry = grid->geometry;
    h->nx = grid->n_x;
    h->ny = grid->n_y;
    h->nz = grid->n_z;
    h->nrhs = grid->nrhs;
    h->plane = plane;
    h->vol = plane * grid->n_z;
    h->ntot = h->vol * grid->nrhs;
    // the panel's edge faces carry weight 0, so its axes are walked as if periodic
    h->periodic_y = grid->geometry == PCG_GEOM_LATLON ? 0 : 1;
    const bool field = coeffs->alpha_e || coeffs->alpha_n;
    h->cls_mode = (field || grid->geometry == PCG_GEOM_CUBED_PANEL) ? 2 : (grid->geometry == PCG_GEOM_LATLON ? 1 : 0);
    h->ncls = h->cls_mode == 0 ? 1 : (h->cls_mode == 1 ? h->ny : (int)plane);
    if (opts) {
        h->precision = opts->precision;
        if (opts->inner_tol > 0) h->inner_tol = opts->inner_tol;
        if (opts->inner_maxit > 0) h->inner_maxit = opts->inner_maxit;
        if (opts->max_outer > 0) h->max_outer = opts->max_outer;
        if (opts->passes_per_launch > 0) h->ppl = opts->passes_per_launch;
        h->stream = (cudaStream_t)opts->stream;
        h->precond = opts->preconditioner;
        if (opts->algorithm != PCG_ALG_INTERLEAVED && opts->algorithm != PCG_ALG_SINGLE_REDUCTION) {
            delete h;
            return fail(nullptr, PCG_ERR_INVALID_ARG, "unknown algorithm");
        }
        h->alg_sr = opts->algorithm == PCG_ALG_SINGLE_REDUCTION;
    }
    if (h->precision != PCG_FP64 && h->precision != PCG_MIXED) {
        delete h;
        return fail(nullptr, PCG_ERR_INVALID_ARG, "unknown precision");
    }
    if (h->precond != PCG_PREC_LINE && h->precond != PCG_PREC_MULTIGRID && h->precond != PCG_PREC_MULTIGRID_F32) {
        delete h;
        return fail(nullptr, PCG_ERR_INVALID_ARG, "unknown preconditioner");
    }
    h->mg_f32 = h->precond == PCG_PREC_MULTIGRID_F32;
    if (h->mg_f32) h->precond = PCG_PREC_MULTIGRID;
    // A multigrid-preconditioned solve takes about 20 passes, and the two
    // graph launches in flight at its end run their remaining passes as
    // early exits, about 30 kernels each: 4 passes per launch instead of 16
    // cut those to a few (a launch of 4 passes still outlasts the host's poll)
    if (h->precond == PCG_PREC_MULTIGRID && !(opts && opts->passes_per_launch > 0)) h->ppl = 4;
    if (h->precond == PCG_PREC_MULTIGRID && h->precision != PCG_FP64) {
        delete h;
        return fail(nullptr, PCG_ERR_INVALID_ARG, "the multigrid preconditioner is available with PCG_FP64 only");
    }
    if (h->alg_sr && (h->precond != PCG_PREC_LINE || h->mg_f32 || h->nz > pcg::SR_MAX_NZ || h->nrhs > 65535 ||
                      (h->ny + pcg::SR_TY - 1) / pcg::SR_TY > 65535)) {
        delete h;
        return fail(nullptr, PCG_ERR_INVALID_ARG,
                    "PCG_ALG_SINGLE_REDUCTION needs PCG_PREC_LINE and n_z <= " + std::to_string(pcg::SR_MAX_NZ));
    }
    if (const char* e = std::getenv("PCG_MG_TAIL")) h->mg_tail_cols = std::atoll(e);                  // 0: no k_mg_tail
    if (const char* e = std::getenv("PCG_MG_QUAD")) h->mg_quad = std::atoll(e);                       // 0: no k_mg_resid4
    h->rhs_stats.assign(h->nrhs, pcg_stats_t{});
    if (const char* tr = std::getenv("PCG_TRACE")) h->trace = std::atoi(tr);
    h->block = dim3(BX, BY, 1);
    h->grid = dim3((h->nx + BX - 1) / BX, (h->ny + BY - 1) / BY, h->nrhs);
    h->nblocks = (int)(h->grid.x * h->grid.y);
    if (h->alg_sr) {
        // the tile of the precision the single-reduction sweep runs in (the
        // whole solve in FP64, the inner solve of the mixed form in FP32)
        const int tx = h->precision == PCG_MIXED ? pcg::SrTile<float>::TX : pcg::SrTile<double>::TX;
        h->grid_sr = dim3((h->nx + tx - 1) / tx, (h->ny + pcg::SR_TY - 1) / pcg::SR_TY, h->nrhs);
        h->nblk_sr = (int)(h->grid_sr.x * h->grid_sr.y);
        h->ppl += h->ppl & 1;   // passes alternate the r, s, w buffers: an even count ends where it began
    }
    {
        // The one-thread-per-column sweeps keep every tile resident at once, so
        // the SM with the most tiles sets their duration: take the tile height
        // (4, 2 or 1 rows of 32 columns) that spreads the tiles most evenly
        // over the SMs (65 536 columns: 512 tiles of 4 rows put 4 on some SMs
        // and 3.37 on average; 1024 tiles of 2 rows, 7 against 6.74).
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 1;
        int by = BY;
        double best = -1.0;
        for (int cand : {4, 2, 1}) {
            if ((h->ny + cand - 1) / cand > 65535) continue;   // grid y limit
            const long long tiles = (long long)((h->nx + BX - 1) / BX) * ((h->ny + cand - 1) / cand) * h->nrhs;
            const long long per_sm = (tiles + sms - 1) / sms;
            const double bal = (double)tiles / (double)(per_sm * sms);
            if (bal > best + 0.01) { best = bal; by = cand; }
        }
        if (const char* e = std::getenv("PCG_COL_BY")) {       // experiments: fixed tile height
            const int v = std::atoi(e);
            if (v == 1 || v == 2 || v == 4) by = v;
        }
        h->block_c = dim3(BX, by, 1);
        // PCG_SPMV_KSPLIT=2 splits every column of the SpMV sweep in two parts
        // (twice the threads); measured 5 % slower at 256^2 x 128 and no faster
        // elsewhere, so one part is the default.
        h->ksplit = 1;
        // u, p, q of the next 4 levels loaded before the current ones are stored:
        // 295.6 -> 288.9 us at 256^2 x 128, 4231 -> 4058 us at 1024^2 x 128
        if (const char* e = std::getenv("PCG_SPMV_PIPE")) h->spmv_pipe = std::atoi(e) ? 1 : 0;   // experiments
        if (const char* e = std::getenv("PCG_SPMV_KSPLIT")) {  // experiments: 1 or 2
            const int v = std::atoi(e);
            if (v == 1 || (v == 2 && h->nz >= 2 && (long long)h->nrhs * 2 <= 65535)) h->ksplit = v;
        }
        h->grid_c = dim3((h->nx + BX - 1) / BX, (h->ny + by - 1) / by, h->nrhs);
        h->nblk_c = (int)(h->grid_c.x * h->grid_c.y);
    }
    // Sweep variants: the FP32 sweeps split every column into chunks of 16 or 32
    // levels (up to 8 chunks; HBM latency needs the extra parallelism), the FP64
    // sweeps keep one thread per column (they are bound by the FP64 pipe, which
    // the chunk corrections would load further).  PCG_KERNELS=column|chunked
    // overrides both.
    h->chunked32 = h->nz <= 256 ? 1 : 0;
    h->chunked64 = 0;
    if (const char* kv = std::getenv("PCG_KERNELS")) {
        if (!std::strcmp(kv, "column")) h->chunked32 = h->chunked64 = 0;
        if (!std::strcmp(kv, "chunked") && h->nz <= 256) h->chunked32 = h->chunked64 = 1;
    }
    h->lz_a = h->nz <= 128 ? 16 : 32;
    const int nch_a = (h->nz + h->lz_a - 1) / h->lz_a;
    h->block_a = dim3(32, nch_a, 1);
    h->grid_a = dim3((h->nx + 31) / 32, h->ny, h->nrhs);
    h->nblk_a = (int)(h->grid_a.x * h->grid_a.y);
    h->lz_b = 16;
    if (const char* e = std::getenv("PCG_PDL")) h->pdl = std::atoi(e) ? 1 : 0;
    h->nch_b = (h->nz + h->lz_b - 1) / h->lz_b;
    h->block_b = dim3(BX, BY, 1);
    h->grid_b = dim3((h->nx + BX - 1) / BX, (h->ny + BY - 1) / BY, h->nrhs * h->nch_b);
    h->nblk_b = (int)(h->grid_b.x * h->grid_b.y) * h->nch_b;
    if ((long long)h->nrhs * h->nch_b > 65535 || h->grid_a.y > 65535) h->chunked32 = h->chunked64 = 0;
    // FP32 SpMV sweep without TMA: chunked while the grid has few columns
    // (65536 columns: 93 us vs 123 us per sweep at 128 levels); one thread per
    // column once there are enough columns to hide latency (2^20 columns:
    // 966 us vs 1300 us).
    h->spmv32 = (h->chunked32 && h->plane * (long long)h->nrhs < (1LL << 19)) ? 1 : 0;
    h->spmv64 = h->chunked64 ? 1 : 0;
    // TMA-staged FP32 SpMV sweep (k_sweep_spmv_tma): tiles of 32 x 8 columns x
    // 16 levels; the tensor maps need rows of a multiple of 16 bytes (n_x % 4 == 0)
    // TMA SpMV tiles of 32 x 4 columns (5 blocks of 42 KB per SM): 65.3 us at
    // 256^2 x 128 and 848 us at 1024^2 x 128, against 71.4 and 908 us for
    // 32 x 8 tiles (2 blocks of 78 KB per SM)
    if (const char* e = std::getenv("PCG_TMA_BY")) h->tma_by = std::atoi(e) == 8 ? 8 : 4;   // experiments
    h->block_t = dim3(BX, h->tma_by, 1);
    h->grid_t = dim3((h->nx + BX - 1) / BX, (h->ny + h->tma_by - 1) / h->tma_by, h->nrhs * h->nch_b);
    h->nblk_t = (int)(h->grid_t.x * h->grid_t.y) * h->nch_b;
    const bool tma_ok = h->lz_b == TMA_LZ && h->nx % 4 == 0 && (long long)h->nrhs * h->nch_b <= 65535 &&
                        (long long)h->nz * h->nrhs < (1LL << 31);
    // the persistent two-stage TMA sweep wherever it applies: 54 us at
    // 256^2 x 128, 648 us at 1024^2 x 128, 4.50 ms for 16 rhs of 1440 x 640 x 64
    // (4.3, 5.8, 5.9 TB/s), against 58 us, 832 us and 5.11 ms single-stage;
    // with two threads per column 51 us and 621 us
    if (tma_ok) h->spmv32 = 4;
    // TMA-pipelined FP32 preconditioner sweep: items of prec_R rows of 32
    // columns (prec_R x chunks <= 8 warps), same eligibility plus the chunked form
    {
        const int nch_p = (h->nz + h->lz_a - 1) / h->lz_a;
        h->prec_R = std::max(1, 8 / nch_p);
        h->prec_gx = (h->nx + BX - 1) / BX;
        h->prec_items = h->prec_gx * ((h->ny + h->prec_R - 1) / h->prec_R);
        const bool ptma_ok = h->chunked32 && h->lz_a == 16 && nch_p <= 8 && h->nx % 4 == 0 && h->nrhs <= 65535 &&
                             (long long)h->nz * h->nrhs < (1LL << 31);
        h->prec32 = ptma_ok ? 2 : 0;   // 256x256x128: 52.9 -> 50.8 us; 512x512x64: 93.8 -> 85.2 us
        if (const char* pv = std::getenv("PCG_PREC")) {            // experiments: chunked|tma|tma-generic
            if (!std::strcmp(pv, "chunked")) h->prec32 = 0;
            if (!std::strcmp(pv, "tma")) h->prec32 = ptma_ok ? 2 : 0;
            if (!std::strcmp(pv, "tma-generic")) {                   // no per-level tables (tests)
                h->prec32 = ptma_ok ? 2 : 0;
                h->prec_generic = 1;
            }
        }
    }
    if (const char* sv = std::getenv("PCG_SPMV")) {            // experiments: column|chunked|tma|tma2
        const int m = !std::strcmp(sv, "chunked") ? 1 : (!std::strcmp(sv, "tma") ? 3 : (!std::strcmp(sv, "tma2") ? 4 : 0));
        if (h->nz <= 256 && (long long)h->nrhs * h->nch_b <= 65535) {
            h->spmv32 = (m >= 3 && !tma_ok) ? 1 : m;
            if (m < 3) h->spmv64 = m;
        }
    }

    auto bail = [&](int rc) {
        g_create_error = h->err;
        g_null_error = nullptr;
        pcg_destroy(h);
        return rc;
    };
    HostTables t;
    int rc = build_tables(h, grid, coeffs, t);
    if (rc) return bail(rc);
    cudaError_t e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { h->err = std::string("cudaStreamCreate: ") + cudaGetErrorString(e); return bail(PCG_ERR_CUDA); }
    for (auto& ev : h->ev) {
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) { h->err = std::string("cudaEventCreate: ") + cudaGetErrorString(e); return bail(PCG_ERR_CUDA); }
    }
    if ((rc = dmalloc(h, &h->st, h->nrhs))) return bail(rc);
    if ((rc = dmalloc(h, &h->st_in, h->nrhs))) return bail(rc);
    if ((rc = dmalloc(h, &h->d_active, h->nrhs))) return bail(rc);
    if ((rc = dmalloc(h, &h->partials, (size_t)h->nrhs * std::max(std::max(std::max(h->nblocks, 2 * h->nblk_c), h->prec_items), std::max(std::max(std::max(h->nblk_a, h->nblk_b), 2 * h->nblk_t), h->nblk_sr)) * 4))) return bail(rc);
    if ((rc = dmalloc(h, &h->counters, h->nrhs))) return bail(rc);
    e = cudaMemsetAsync(h->counters, 0, sizeof(unsigned) * h->nrhs, h->stream);
    if (e != cudaSuccess) { h->err = std::string("cudaMemset: ") + cudaGetErrorString(e); return bail(PCG_ERR_CUDA); }
    e = cudaMallocHost((void**)&h->h_st, sizeof(SolveState) * 2 * h->nrhs);
    if (e != cudaSuccess) { h->h_st = nullptr; h->err = "cudaMallocHost failed"; return bail(PCG_ERR_OOM); }
    if ((rc = upload_tables(h, t))) return bail(rc);
    if (h->precond == PCG_PREC_MULTIGRID && (rc = build_hierarchy(h, grid, coeffs))) return bail(rc);
    if (h->precond == PCG_PREC_MULTIGRID && h->mg_tail_cols > 0 && !tail_ready(h)) h->mg_tail_cols = 0;
    *out = h;
    return PCG_OK;
}

int pcg_solve(pcg_t h, const double* b, double* x, double tol, int maxit, pcg_stats_t* stats) {
    if (!h) return fail(nullptr, PCG_ERR_INVALID_ARG, "handle is NULL");
    if (!b || !x) return fail(h, PCG_ERR_INVALID_ARG, "b and x are required");
    if (!(tol >= 0.0) || maxit < 0) return fail(h, PCG_ERR_INVALID_ARG, "tol must be >= 0 and maxit >= 0");
    const double t0 = now_ms();
    int rc = h->precision == PCG_MIXED ? solve_mixed(h, b, x, tol, maxit, stats) : solve_fp64(h, b, x, tol, maxit, stats);
    if (rc == PCG_ERR_CUDA || rc == PCG_ERR_OOM || rc == PCG_ERR_INVALID_ARG) return rc;
    summarise(h, stats, rc, t0);
    return rc;
}

int pcg_solve_host(pcg_t h, const double* b_host, double* x_host, double tol, int maxit, pcg_stats_t* stats) {
    if (!h) return fail(nullptr, PCG_ERR_INVALID_ARG, "handle is NULL");
    if (!b_host || !x_host) return fail(h, PCG_ERR_INVALID_ARG, "b and x are required");
    const double t0 = now_ms();
    int rc;
    if (!h->hb) {
        if ((rc = dmalloc(h, &h->hb, (size_t)h->ntot))) return rc;
        if ((rc = dmalloc(h, &h->hx, (size_t)h->ntot))) return rc;
    }
    const size_t nb = sizeof(double) * h->ntot;
    PCG_CK(h, cudaMemcpyAsync(h->hb, b_host, nb, cudaMemcpyHostToDevice, h->stream));
    PCG_CK(h, cudaMemcpyAsync(h->hx, x_host, nb, cudaMemcpyHostToDevice, h->stream));
    rc = h->precision == PCG_MIXED ? solve_mixed(h, h->hb, h->hx, tol, maxit, stats)
                                   : solve_fp64(h, h->hb, h->hx, tol, maxit, stats);
    if (rc == PCG_ERR_CUDA || rc == PCG_ERR_OOM || rc == PCG_ERR_INVALID_ARG) return rc;
    PCG_CK(h, cudaMemcpyAsync(x_host, h->hx, nb, cudaMemcpyDeviceToHost, h->stream));
    PCG_CK(h, cudaStreamSynchronize(h->stream));
    summarise(h, stats, rc, t0);
    return rc;
}

int pcg_rhs_stats(pcg_t h, int rhs, pcg_stats_t* stats) {
    if (!h || !stats) return fail(h, PCG_ERR_INVALID_ARG, "handle and stats are required");
    if (rhs < 0 || rhs >= h->nrhs) return fail(h, PCG_ERR_INVALID_ARG, "rhs out of range");
    *stats = h->rhs_stats[rhs];
    return PCG_OK;
}

int pcg_apply_A(pcg_t h, const double* x, double* y) {
    if (!h) return fail(nullptr, PCG_ERR_INVALID_ARG, "handle is NULL");
    if (!x || !y) return fail(h, PCG_ERR_INVALID_ARG, "x and y are required");
    pcg::k_apply<double><<<h->grid, h->block, 0, h->stream>>>(h->view64(), x, y);
    PCG_CK(h, cudaGetLastError());
    return PCG_OK;
}

int pcg_precond(pcg_t h, const double* r, double* z) {
    if (!h) return fail(nullptr, PCG_ERR_INVALID_ARG, "handle is NULL");
    if (!r || !z) return fail(h, PCG_ERR_INVALID_ARG, "r and z are required");
    if (h->precond == PCG_PREC_MULTIGRID && h->mg_f32) {
        const dim3 g = elem_grid(h->vol, h->nrhs);
        pcg::k_mg_convert<double, float><<<g, 256, 0, h->stream>>>(r, h->mg_r0f, h->vol, h->nrhs, h->mg_free);
        launch_vcycle<float>(h, h->stream, h->mg_free, h->mg_r0f, h->mg_z0f, h->mg_t0f);
        pcg::k_mg_convert<float, double><<<g, 256, 0, h->stream>>>(h->mg_z0f, z, h->vol, h->nrhs, h->mg_free);
    } else if (h->precond == PCG_PREC_MULTIGRID)
        launch_vcycle<double>(h, h->stream, h->mg_free, r, z, h->mg_t0);
    else
        pcg::k_precond<double><<<h->grid, h->block, 0, h->stream>>>(h->view64(), r, z);
    PCG_CK(h, cudaGetLastError());
    return PCG_OK;
}

int pcg_apply_A_f32(pcg_t h, const float* x, float* y) {
    if (!h) return fail(nullptr, PCG_ERR_INVALID_ARG, "handle is NULL");
    if (!x || !y) return fail(h, PCG_ERR_INVALID_ARG, "x and y are required");
    pcg::k_apply<float><<<h->grid, h->block, 0, h->stream>>>(h->view32(), x, y);
    PCG_CK(h, cudaGetLastError());
    return PCG_OK;
}

int pcg_precond_f32(pcg_t h, const float* r, float* z) {
    if (!h) return fail(nullptr, PCG_ERR_INVALID_ARG, "handle is NULL");
    if (!r || !z) return fail(h, PCG_ERR_INVALID_ARG, "r and z are required");
    pcg::k_precond<float><<<h->grid, h->block, 0, h->stream>>>(h->view32(), r, z);
    PCG_CK(h, cudaGetLastError());
    return PCG_OK;
}

int pcg_time_sweeps(pcg_t h, const double* b, int precision, int passes, double* ms_prec, double* ms_spmv) {
    if (!h) return fail(nullptr, PCG_ERR_INVALID_ARG, "handle is NULL");
    if (!b || !ms_prec || !ms_spmv || passes < 1) return fail(h, PCG_ERR_INVALID_ARG, "b, outputs and passes >= 1 required");
    if (precision != PCG_FP64 && precision != PCG_MIXED) return fail(h, PCG_ERR_INVALID_ARG, "unknown precision");
    int rc;
    if ((rc = ensure_ws64(h))) return rc;
    if (precision == PCG_MIXED && (rc = ensure_ws32(h))) return rc;
    cudaStream_t s = h->stream;
    const OpView<double> v = h->view64();
    std::vector<cudaEvent_t> ev(3);
    for (auto& e : ev) PCG_CK(h, cudaEventCreate(&e));
    double tp = 0.0, ts = 0.0;
    PCG_CK(h, cudaMemsetAsync(h->z64, 0, sizeof(double) * h->ntot, s));   // x0 = 0
    pcg::k_init_state<<<(h->nrhs + 63) / 64, 64, 0, s>>>(h->st, h->nrhs, 0.0, passes, nullptr);
    if (precision == PCG_FP64) {
        pcg::k_residual<double><<<h->grid, h->block, 0, s>>>(v, b, h->z64, h->u64, h->r64, h->st, h->partials,
                                                            h->counters, h->nblocks, 0);
        PCG_CK(h, cudaMemsetAsync(h->p64, 0, sizeof(double) * h->ntot, s));
        PCG_CK(h, cudaMemsetAsync(h->q64, 0, sizeof(double) * h->ntot, s));
    } else {
        pcg::k_residual<float><<<h->grid, h->block, 0, s>>>(v, b, h->z64, nullptr, h->r32, h->st, h->partials,
                                                           h->counters, h->nblocks, 3);
        pcg::k_init_state<<<(h->nrhs + 63) / 64, 64, 0, s>>>(h->st_in, h->nrhs, 0.0, passes, nullptr);
        PCG_CK(h, cudaMemsetAsync(h->u32, 0, sizeof(float) * h->ntot, s));
        PCG_CK(h, cudaMemsetAsync(h->p32, 0, sizeof(float) * h->ntot, s));
        PCG_CK(h, cudaMemsetAsync(h->q32, 0, sizeof(float) * h->ntot, s));
    }
    PCG_CK(h, cudaGetLastError());
    const OpView<float> v32 = h->view32();
    for (int i = 0; i < passes; ++i) {
        PCG_CK(h, cudaEventRecord(ev[0], s));
        if (precision == PCG_FP64)
            launch_prec<double>(h, s, v, h->r64, h->q64, h->z64, h->st);
        else
            launch_prec<float>(h, s, v32, h->r32, h->q32, h->z32, h->st_in);
        PCG_CK(h, cudaEventRecord(ev[1], s));
        if (precision == PCG_FP64)
            launch_spmv<double>(h, s, v, h->u64, h->p64, h->q64, h->z64, h->st);
        else
            launch_spmv<float>(h, s, v32, h->u32, h->p32, h->q32, h->z32, h->st_in);
        PCG_CK(h, cudaEventRecord(ev[2], s));
        PCG_CK(h, cudaGetLastError());
        PCG_CK(h, cudaEventSynchronize(ev[2]));
        float a = 0.f, c = 0.f;
        PCG_CK(h, cudaEventElapsedTime(&a, ev[0], ev[1]));
        PCG_CK(h, cudaEventElapsedTime(&c, ev[1], ev[2]));
        tp += a;
        ts += c;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    *ms_prec = tp / passes;
    *ms_spmv = ts / passes;
    return PCG_OK;
}

int pcg_time_passes(pcg_t h, const double* b, int precision, int passes, double* ms_per_pass) {
    if (!h) return fail(nullptr, PCG_ERR_INVALID_ARG, "handle is NULL");
    if (!b || !ms_per_pass || passes < 1) return fail(h, PCG_ERR_INVALID_ARG, "b, ms_per_pass and passes >= 1 required");
    if (precision != PCG_FP64 && precision != PCG_MIXED) return fail(h, PCG_ERR_INVALID_ARG, "unknown precision");
    int rc;
    if ((rc = ensure_ws64(h))) return rc;
    if (precision == PCG_MIXED && (rc = ensure_ws32(h))) return rc;
    cudaStream_t s = h->stream;
    const OpView<double> v = h->view64();
    const OpView<float> v32 = h->view32();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PCG_CK(h, cudaEventCreate(&e0));
    PCG_CK(h, cudaEventCreate(&e1));
    PCG_CK(h, cudaMemsetAsync(h->z64, 0, sizeof(double) * h->ntot, s));   // x0 = 0
    pcg::k_init_state<<<(h->nrhs + 63) / 64, 64, 0, s>>>(h->st, h->nrhs, 0.0, passes, nullptr);
    if (precision == PCG_FP64) {
        pcg::k_residual<double><<<h->grid, h->block, 0, s>>>(v, b, h->z64, h->u64, h->r64, h->st, h->partials,
                                                            h->counters, h->nblocks, 0);
        PCG_CK(h, cudaMemsetAsync(h->p64, 0, sizeof(double) * h->ntot, s));
        PCG_CK(h, cudaMemsetAsync(h->q64, 0, sizeof(double) * h->ntot, s));
    } else {
        pcg::k_residual<float><<<h->grid, h->block, 0, s>>>(v, b, h->z64, nullptr, h->r32, h->st, h->partials,
                                                           h->counters, h->nblocks, 3);
        pcg::k_init_state<<<(h->nrhs + 63) / 64, 64, 0, s>>>(h->st_in, h->nrhs, 0.0, passes, nullptr);
        PCG_CK(h, cudaMemsetAsync(h->u32, 0, sizeof(float) * h->ntot, s));
        PCG_CK(h, cudaMemsetAsync(h->p32, 0, sizeof(float) * h->ntot, s));
        PCG_CK(h, cudaMemsetAsync(h->q32, 0, sizeof(float) * h->ntot, s));
    }
    PCG_CK(h, cudaGetLastError());
    PCG_CK(h, cudaEventRecord(e0, s));
    for (int i = 0; i < passes; ++i) {
        if (precision == PCG_FP64) {
            launch_prec<double>(h, s, v, h->r64, h->q64, h->z64, h->st);
            launch_spmv<double>(h, s, v, h->u64, h->p64, h->q64, h->z64, h->st);
        } else {
            launch_prec<float>(h, s, v32, h->r32, h->q32, h->z32, h->st_in, h->pdl != 0);
            launch_spmv<float>(h, s, v32, h->u32, h->p32, h->q32, h->z32, h->st_in, h->pdl != 0);
        }
    }
    PCG_CK(h, cudaEventRecord(e1, s));
    PCG_CK(h, cudaGetLastError());
    PCG_CK(h, cudaEventSynchronize(e1));
    float ms = 0.f;
    PCG_CK(h, cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_per_pass = ms / passes;
    return PCG_OK;
}

int pcg_sync(pcg_t h) {
    if (!h) return fail(nullptr, PCG_ERR_INVALID_ARG, "handle is NULL");
    PCG_CK(h, cudaStreamSynchronize(h->stream));
    return PCG_OK;
}

size_t pcg_device_bytes(pcg_t h) { return h ? h->bytes : 0; }

long long pcg_kernel_launches(pcg_t h) { return h ? h->launches : 0; }

const char* pcg_last_error(pcg_t h) { return h ? h->err.c_str() : (g_null_error ? g_null_error : g_create_error.c_str()); }

void pcg_destroy(pcg_t h) {
    if (!h) return;
    if (h->stream || h->cap_stream) cudaStreamSynchronize(h->stream);
    for (auto& l : h->mg) {
        for (void* p : {(void*)l.r, (void*)l.z, (void*)l.t, (void*)l.rf, (void*)l.zf, (void*)l.tf})
            if (p) cudaFree(p);
        pcg_destroy(l.h);
    }
    h->mg.clear();
    if (h->mg_t0) cudaFree(h->mg_t0);
    for (void* p : {(void*)h->mg_r0f, (void*)h->mg_z0f, (void*)h->mg_t0f})
        if (p) cudaFree(p);
    if (h->mg_free) cudaFree(h->mg_free);
    if (h->graph64) cudaGraphExecDestroy(h->graph64);
    if (h->graph32) cudaGraphExecDestroy(h->graph32);
    if (h->graph_sr) cudaGraphExecDestroy(h->graph_sr);
    if (h->graph_sr32) cudaGraphExecDestroy(h->graph_sr32);
    for (void* p : {(void*)h->r64b, (void*)h->s64b, (void*)h->w64a, (void*)h->w64b, (void*)h->r32b, (void*)h->s32b,
                    (void*)h->w32a, (void*)h->w32b})
        if (p) cudaFree(p);
    for (void* p : {(void*)h->u64, (void*)h->r64, (void*)h->z64, (void*)h->p64, (void*)h->q64, (void*)h->u32,
                    (void*)h->r32, (void*)h->z32, (void*)h->p32, (void*)h->q32, (void*)h->hb, (void*)h->hx,
                    (void*)h->st, (void*)h->st_in, (void*)h->d_active, (void*)h->partials, (void*)h->counters,
                    h->t64.base, h->t32.base})
        if (p) cudaFree(p);
    if (h->h_st) cudaFreeHost(h->h_st);
    for (auto ev : h->ev)
        if (ev) cudaEventDestroy(ev);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Line preconditioner without any allocation.
//
// For callers that must not allocate device memory at the point of the call:
// real-time loops that cannot afford an allocation's latency or the
// synchronisation a cudaMalloc/cudaFree may imply, and hosts whose device
// memory is owned entirely by another allocator (a framework's caching
// allocator or a fixed budget), so that a library-side cudaMalloc would fail
// or fragment it.  Such callers cannot create a handle at that point, because
// pcg_create allocates.  pcg_precond_noalloc applies the same preconditioner
// as pcg_precond: the operator tables come from the same host routine
// (tables_into) and the factors from the same kernel (k_factors), kept in the
// fixed-size device array below, which every GPU that loads this library
// holds until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocDoubles = size_t(1) << 19;   // 4 MiB of device scratch

__device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];
double g_noalloc_stage[kNoAllocDoubles];              // host staging of the tables (same layout)
constexpr int kNoAllocMaxDevices = 64;
double* g_noalloc_dev_ptr[kNoAllocMaxDevices] = {};   // device address of the scratch, per device
thread_local char g_noalloc_msg[320];                 // error text of this thread's last failed call

int noalloc_fail(int code, const char* msg) {
    std::snprintf(g_noalloc_msg, sizeof g_noalloc_msg, "pcg_precond_noalloc: %s", msg);
    g_null_error = g_noalloc_msg;
    return code;
}

}  // namespace

extern "C" int pcg_precond_noalloc(const pcg_grid_t* grid, const pcg_coeffs_t* coeffs, const double* r, double* z,
                                   void* stream) {
    if (!grid || !coeffs || !r || !z) return noalloc_fail(PCG_ERR_INVALID_ARG, "grid, coeffs, r and z are required");
    if (grid->n_x < 1 || grid->n_y < 1 || grid->n_z < 1 || grid->nrhs < 1)
        return noalloc_fail(PCG_ERR_INVALID_ARG, "n_x, n_y, n_z and nrhs must be >= 1");
    if (grid->nrhs > 65535) return noalloc_fail(PCG_ERR_INVALID_ARG, "nrhs must be <= 65535");
    if (!grid->z_iface || !coeffs->beta_iface) return noalloc_fail(PCG_ERR_INVALID_ARG, "z_iface and beta_iface are required");
    if (!(coeffs->lambda2 >= 0.0) || !std::isfinite(coeffs->lambda2))
        return noalloc_fail(PCG_ERR_INVALID_ARG, "lambda2 must be finite and >= 0");
    const int geo = grid->geometry;
    if (geo != PCG_GEOM_BOX && geo != PCG_GEOM_LATLON && geo != PCG_GEOM_CUBED_PANEL)
        return noalloc_fail(PCG_ERR_INVALID_ARG, "unknown geometry");
    const int nx = grid->n_x, ny = grid->n_y, nz = grid->n_z;
    const size_t nxy = (size_t)nx * ny;
    // factor classes exactly as pcg_create chooses them
    const bool field = coeffs->alpha_e || coeffs->alpha_n;
    const int cls_mode = (field || geo == PCG_GEOM_CUBED_PANEL) ? 2 : (geo == PCG_GEOM_LATLON ? 1 : 0);
    const size_t ncls = cls_mode == 0 ? 1 : (cls_mode == 1 ? (size_t)ny : nxy);
    const size_t na = table_area_len(grid);
    const size_t ntab = 3 * (size_t)nz + na + 2 * nxy;
    const size_t need = ntab + 3 * (size_t)nz * ncls;
    if (need > kNoAllocDoubles) {
        char msg[256];
        std::snprintf(msg, sizeof msg,
                      "this grid needs %zu doubles of tables and factors, the fixed scratch holds %zu "
                      "(use pcg_create and pcg_precond)", need, kNoAllocDoubles);
        return noalloc_fail(PCG_ERR_INVALID_ARG, msg);
    }
    // one-time set-up per device: the device address of the scratch array
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(PCG_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return noalloc_fail(PCG_ERR_INVALID_ARG, "device ordinal out of range");
    if (!g_noalloc_dev_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return noalloc_fail(PCG_ERR_CUDA, cudaGetErrorString(e));
        g_noalloc_dev_ptr[dev] = (double*)p;
    }
    double* d = g_noalloc_dev_ptr[dev];
    // tables (Section 3.1 geometry) into the static host staging buffer, by
    // the routine pcg_create uses
    double* hs = g_noalloc_stage;
    const TableOut tout{hs, hs + nz, hs + 2 * nz, hs + 3 * nz, hs + 3 * nz + na, hs + 3 * nz + na + nxy};
    const char* msg = nullptr;
    double total_mass = 0.0;
    if (tables_into(grid, coeffs, tout, &msg, &total_mass)) return noalloc_fail(PCG_ERR_INVALID_ARG, msg);
    cudaStream_t s = (cudaStream_t)stream;
    // a copy from pageable host memory returns once the staging buffer has been read
    e = cudaMemcpyAsync(d, hs, ntab * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return noalloc_fail(PCG_ERR_CUDA, cudaGetErrorString(e));
    OpView<double> v;
    v.nx = nx;
    v.ny = ny;
    v.nz = nz;
    v.plane = (long long)nxy;
    v.vol = (long long)nxy * nz;
    v.mass = d;
    v.wv = d + nz;
    v.dk = d + 2 * nz;
    v.area = d + 3 * nz;
    v.mue = v.area + na;
    v.mun = v.mue + nxy;
    // the panel's edge faces carry weight 0, so its axes are walked as if periodic (as in pcg_create)
    v.periodic_y = geo == PCG_GEOM_LATLON ? 0 : 1;
    double* fg = d + ntab;
    double* fe = fg + (size_t)nz * ncls;
    double* fc = fe + (size_t)nz * ncls;
    v.fg = fg;
    v.fe = fe;
    v.fc = fc;
    v.cls_mode = cls_mode;
    v.ncls = (int)ncls;
    v.area_percol = geo == PCG_GEOM_CUBED_PANEL ? 1 : 0;
    v.amass = nullptr;
    v.awv = nullptr;
    v.arow_step = 0;
    // the factors are rewritten in full by every call, so nothing left by an
    // earlier call is read
    pcg::k_factors<<<(unsigned)((ncls + 127) / 128), 128, 0, s>>>(v, fg, fe, fc);
    const dim3 block(BX, BY, 1), gridd((nx + BX - 1) / BX, (ny + BY - 1) / BY, grid->nrhs);
    pcg::k_precond<double><<<gridd, block, 0, s>>>(v, r, z);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(PCG_ERR_CUDA, cudaGetErrorString(e));
    return PCG_OK;
}

#include "serve.cuh"
