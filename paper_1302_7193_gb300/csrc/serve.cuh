// Served batch of mixed-precision solves (continuous batching).
//
// A request is one solve A x = b of its own grid, coefficients and
// tolerance.  Submitted requests wait in a FIFO queue and are admitted while
// the device-byte budget and the slot count allow; an admitted request gets
// its tables (Section 3.1 geometry, FP64 Thomas factors) and its vectors in
// one stream-ordered allocation.  Each request runs the mixed-precision
// refinement of pcg_solve: FP64 residual, coarse correction, FP32 inner PCG
// (Algorithm 1), FP64 update.  The inner iterations of all requests that are
// in their inner phase advance together: one CUDA graph holds
// `epochs_per_launch` epochs, an epoch being one launch of k_serve_prec and
// one of k_serve_spmv, persistent kernels that walk the work lists of
// (slot, item) pairs of every such request (preconditioner items: rows of
// 32 columns split into 16-level chunks; SpMV items: 32 x 8-column tiles of
// one 16-level chunk, staged by bulk tensor copies).  Between graph launches the host
// runs the FP64 refinement steps of requests whose inner solve finished,
// retires requests that converged (their x is copied out and their memory
// returned) and admits waiting requests into the freed slots, so new
// requests join the work of the ones already on the GPU.
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <type_traits>
#include <unordered_map>

namespace {

enum ServePhase { RQ_PENDING = 0, RQ_MEASURE = 1, RQ_INNER = 2, RQ_DONE = 3 };

struct ServeReq {
    uint64_t id = 0;
    int phase = RQ_PENDING;
    int slot = -1;
    pcg_grid_t grid{};
    std::vector<double> z_iface, beta, alpha_e, alpha_n;
    double lambda2 = 0.0;
    std::vector<double> b, x;
    double tol = 1e-8;
    void* dmem = nullptr;
    size_t bytes = 0;
    OpView<double> op64{};
    OpView<float> op32{};
    double *xd = nullptr, *bd = nullptr;
    float *u = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    double* partials = nullptr;
    unsigned* counter = nullptr;
    double total_mass = 0.0;
    int gx = 0, gy = 0, ntiles = 0;          // 32 x 4 tiles (residual kernels)
    int nch = 1, rows = 1, colmode = 0, nprec = 0, nspmv = 0;   // served sweep items
    CUtensorMap* tmaps = nullptr;            // device copies of the u, p, q, z maps and the r, q item maps, or null
    int prec_tma = 0;                        // the preconditioner items are staged (maps 4 and 5)
    std::vector<double> hist;
    double bb = 0.0, last_rr = 0.0, floor_rel = 0.0;
    int sweeps = 0, inner_its = 0, status = PCG_NOT_CONVERGED, stag = 0;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    pcg_stats_t mg_stats{};                  // multigrid mode: the solve's statistics
};

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

using ServeSpmvTile = pcg::SpmvTmaTile<pcg::SERVE_LZ, pcg::SERVE_BY>;

}  // namespace

struct pcg_server {
    size_t budget = 0, used = 0;
    int max_slots = 0;
    double inner_tol = 1e-5;
    int inner_maxit = 20000, max_outer = 16, epochs_per_launch = 8;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    cudaMemPool_t pool = nullptr;
    uint64_t next_id = 1;
    std::deque<ServeReq*> pending;
    std::vector<ServeReq*> slot_req;
    std::unordered_map<uint64_t, ServeReq*> reqs;
    pcg::ServeSlot* d_slots = nullptr;
    std::vector<pcg::ServeSlot> h_slots;
    SolveState* d_states = nullptr;     // [max_slots][2]: inner, outer
    SolveState* h_states = nullptr;     // pinned mirror
    int2* d_items = nullptr;            // [2][items_cap]: preconditioner items, then SpMV items
    int* d_nitems = nullptr;            // [2]
    int2* h_items = nullptr;            // pinned mirror
    int* h_nitems = nullptr;            // pinned [2]
    int* d_one = nullptr;
    int* d_inner = nullptr;             // [max_slots]: 1 while the slot's request is in its inner phase
    int* h_inner = nullptr;             // pinned mirror
    unsigned* d_fetch = nullptr;        // [epochs_per_launch][2]: next item of each epoch's two launches
    int items_cap = 0;
    bool items_dirty = true;
    cudaGraphExec_t graph = nullptr;
    int blocks_prec = 152 * 3, blocks_spmv = 152 * 2;   // persistent grids (resident blocks on every SM)
    long long active_unknowns = 0;      // unknowns of the admitted requests
    long long epochs = 0, launches = 0, retired = 0;
    int trace = 0;                      // PCG_TRACE=1: refinement history per request on stderr
    std::string err = "no error";
    // multigrid mode (opts->preconditioner == PCG_PREC_MULTIGRID_F32, serve_mg.cuh): worker threads
    int mode = 0;                       // 0: batched line-preconditioned mixed solves; 1: multigrid workers
    int device = 0;
    std::vector<std::thread> workers;
    std::mutex mu;                      // mode 1: guards pending, reqs, the requests' phases, used, busy
    std::condition_variable cv_work, cv_done;
    bool stopping = false;
    int busy = 0;                       // mode 1: requests being solved
};

namespace {

int sfail(pcg_server_t s, int code, const std::string& msg) {
    if (s) {
        s->err = msg;
    } else {
        g_create_error = msg;
        g_null_error = nullptr;
    }
    return code;
}

#define SRV_CK(s, call)                                                                       \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            int code_ = (e_ == cudaErrorMemoryAllocation) ? PCG_ERR_OOM : PCG_ERR_CUDA;       \
            return sfail(s, code_, std::string(#call) + ": " + cudaGetErrorString(e_));       \
        }                                                                                     \
    } while (0)

// Bytes one request needs on the device (tables in both precisions, FP64 x
// and b, five FP32 inner vectors, partials and the arrival counter).
int serve_cls_mode(const pcg_grid_t& g, bool field) {
    return (field || g.geometry == PCG_GEOM_CUBED_PANEL) ? 2 : (g.geometry == PCG_GEOM_LATLON ? 1 : 0);
}

size_t area_count(const pcg_grid_t& g) {
    return g.geometry == PCG_GEOM_CUBED_PANEL ? (size_t)g.n_x * g.n_y : (size_t)g.n_y;
}

// Work items of a request in the served sweeps (see k_serve_prec / k_serve_spmv).
struct ServeItems {
    int gx, nch, rows, colmode, nprec, nspmv;
};

ServeItems serve_items(const pcg_grid_t& g) {
    ServeItems it;
    it.gx = (g.n_x + BX - 1) / BX;
    it.nch = (g.n_z + pcg::SERVE_LZ - 1) / pcg::SERVE_LZ;
    it.colmode = it.nch > 8 ? 1 : 0;
    it.rows = it.colmode ? 8 : 8 / it.nch;
    it.nprec = it.gx * ((g.n_y + it.rows - 1) / it.rows);
    it.nspmv = it.gx * ((g.n_y + pcg::SERVE_BY - 1) / pcg::SERVE_BY) * it.nch;
    return it;
}

size_t request_bytes(const pcg_grid_t& g, int cls_mode) {
    const size_t nx = g.n_x, ny = g.n_y, nz = g.n_z, nxy = nx * ny, vol = nxy * nz;
    const size_t ncls = cls_mode == 0 ? 1 : (cls_mode == 1 ? ny : nxy);
    const size_t ntab = 3 * nz + area_count(g) + 2 * nxy + 2 * nz * ncls;
    const size_t ntiles = ((nx + BX - 1) / BX) * ((ny + BY - 1) / BY);
    const ServeItems it = serve_items(g);
    const size_t nparts = std::max(ntiles, (size_t)std::max(it.nprec, it.nspmv));
    return align_up(ntab * 8) + align_up(ntab * 4) + 2 * align_up(vol * 8) + 5 * align_up(vol * 4) +
           align_up(nparts * 4 * 8) + align_up(6 * sizeof(CUtensorMap)) + align_up(5 * nz * 4) + 256;
}

int admit(pcg_server_t s, ServeReq* q) {
    pcg_grid_t g = q->grid;
    g.z_iface = q->z_iface.data();
    pcg_coeffs_t c{};
    c.beta_iface = q->beta.data();
    c.alpha_e = q->alpha_e.empty() ? nullptr : q->alpha_e.data();
    c.alpha_n = q->alpha_n.empty() ? nullptr : q->alpha_n.data();
    c.lambda2 = q->lambda2;
    HostTables t;
    std::string err;
    int rc = build_tables_core(&g, &c, t, err, q->total_mass);
    if (rc) return sfail(s, rc, err);
    const int cls_mode = serve_cls_mode(g, c.alpha_e || c.alpha_n);
    const size_t nx = g.n_x, ny = g.n_y, nz = g.n_z, nxy = nx * ny, vol = nxy * nz;
    const size_t ncls = cls_mode == 0 ? 1 : (cls_mode == 1 ? ny : nxy);
    const size_t na = area_count(g);
    const size_t ntab = 3 * nz + na + 2 * nxy + 2 * nz * ncls;
    q->gx = (int)((nx + BX - 1) / BX);
    q->gy = (int)((ny + BY - 1) / BY);
    q->ntiles = q->gx * q->gy;
    q->bytes = request_bytes(g, cls_mode);
    SRV_CK(s, cudaMallocFromPoolAsync(&q->dmem, q->bytes, s->pool, s->stream));
    char* m = (char*)q->dmem;
    double* t64 = (double*)m;
    m += align_up(ntab * 8);
    float* t32 = (float*)m;
    m += align_up(ntab * 4);
    q->xd = (double*)m;
    m += align_up(vol * 8);
    q->bd = (double*)m;
    m += align_up(vol * 8);
    float** fv[5] = {&q->u, &q->r, &q->z, &q->p, &q->q};
    for (auto v : fv) {
        *v = (float*)m;
        m += align_up(vol * 4);
    }
    const ServeItems its = serve_items(g);
    q->nch = its.nch; q->rows = its.rows; q->colmode = its.colmode; q->nprec = its.nprec; q->nspmv = its.nspmv;
    q->partials = (double*)m;
    m += align_up((size_t)std::max(q->ntiles, std::max(q->nprec, q->nspmv)) * 4 * 8);
    q->tmaps = (CUtensorMap*)m;             // 256-byte aligned like every carved region
    m += align_up(6 * sizeof(CUtensorMap));
    float* ptab = (float*)m;
    m += align_up(5 * nz * 4);
    q->counter = (unsigned*)m;
    // tables: same carving as a solver handle
    auto carve = [&](auto& op, auto* base) {
        using T = std::remove_pointer_t<decltype(base)>;
        size_t off = 0;
        auto nxt = [&](size_t n) { T* p = base + off; off += n; return p; };
        op.nx = (int)nx; op.ny = (int)ny; op.nz = (int)nz;
        op.plane = (long long)nxy; op.vol = (long long)vol;
        op.mass = nxt(nz); op.wv = nxt(nz); op.dk = nxt(nz); op.area = nxt(na);
        op.mue = nxt(nxy); op.mun = nxt(nxy);
        op.fg = nxt(nz * ncls); op.fe = nxt(nz * ncls); op.fc = nullptr;   // served sweeps are FP32
        op.periodic_y = g.geometry == PCG_GEOM_LATLON ? 0 : 1;
        op.cls_mode = cls_mode; op.ncls = (int)ncls;
        op.area_percol = g.geometry == PCG_GEOM_CUBED_PANEL ? 1 : 0;
        op.amass = nullptr; op.awv = nullptr; op.arow_step = 0;
    };
    carve(q->op64, t64);
    carve(q->op32, t32);
    cudaStream_t st = s->stream;
    SRV_CK(s, cudaMemcpyAsync((void*)q->op64.mass, t.mass.data(), nz * 8, cudaMemcpyHostToDevice, st));
    SRV_CK(s, cudaMemcpyAsync((void*)q->op64.wv, t.wv.data(), nz * 8, cudaMemcpyHostToDevice, st));
    SRV_CK(s, cudaMemcpyAsync((void*)q->op64.dk, t.dk.data(), nz * 8, cudaMemcpyHostToDevice, st));
    SRV_CK(s, cudaMemcpyAsync((void*)q->op64.area, t.area.data(), na * 8, cudaMemcpyHostToDevice, st));
    SRV_CK(s, cudaMemcpyAsync((void*)q->op64.mue, t.mue.data(), nxy * 8, cudaMemcpyHostToDevice, st));
    SRV_CK(s, cudaMemcpyAsync((void*)q->op64.mun, t.mun.data(), nxy * 8, cudaMemcpyHostToDevice, st));
    pcg::k_factors<<<(unsigned)((ncls + 127) / 128), 128, 0, st>>>(q->op64, (double*)q->op64.fg, (double*)q->op64.fe,
                                                                    nullptr);
    pcg::k_to_float<<<256, 256, 0, st>>>(t64, t32, (long long)ntab);
    // one factor set and chunked preconditioner items: the chunk-carry tables
    const bool tab = cls_mode == 0 && !q->colmode && nz % pcg::SERVE_LZ == 0 && q->rows <= 4;
    if (tab) pcg::k_build_prec_tab<<<1, 256, 0, st>>>(q->op32, ptab);
    SRV_CK(s, cudaMemcpyAsync(q->bd, q->b.data(), vol * 8, cudaMemcpyHostToDevice, st));
    SRV_CK(s, cudaMemsetAsync(q->xd, 0, vol * 8, st));
    SRV_CK(s, cudaMemsetAsync(q->counter, 0, sizeof(unsigned), st));
    {
        // tensor maps of the SpMV sweep's staged tiles (boxes as k_sweep_spmv_tma)
        // and of the preconditioner items' r and q (32 columns x rows x all
        // chunks); without them the threads stage the tiles and read r, q
        CUtensorMap hm[6];
        const unsigned zx = BX + 2 * pcg::TMA_HALO_X;
        const bool ok = encode_map_dims(&hm[0], q->u, nx, ny, nz, BX, pcg::SERVE_BY, pcg::SERVE_LZ) &&
                        encode_map_dims(&hm[1], q->p, nx, ny, nz, BX, pcg::SERVE_BY, pcg::SERVE_LZ) &&
                        encode_map_dims(&hm[2], q->q, nx, ny, nz, BX, pcg::SERVE_BY, pcg::SERVE_LZ) &&
                        encode_map_dims(&hm[3], q->z, nx, ny, nz, zx, pcg::SERVE_BY + 2, pcg::SERVE_LZ + 2);
        const unsigned pz = (unsigned)(q->nch * pcg::SERVE_LZ);
        q->prec_tma = ok && !q->colmode && (unsigned)q->rows * pz <= (unsigned)(8 * pcg::SERVE_LZ) &&
                      encode_map_dims(&hm[4], q->r, nx, ny, nz, BX, (unsigned)q->rows, pz) &&
                      encode_map_dims(&hm[5], q->q, nx, ny, nz, BX, (unsigned)q->rows, pz);
        if (ok) {
            // pageable source: the call returns once the maps have been staged
            SRV_CK(s, cudaMemcpyAsync(q->tmaps, hm, sizeof(hm), cudaMemcpyHostToDevice, st));
        } else {
            q->tmaps = nullptr;
            q->prec_tma = 0;
        }
    }
    SRV_CK(s, cudaGetLastError());
    s->launches += 2;
    // slot
    int slot = -1;
    for (int i = 0; i < s->max_slots; ++i)
        if (!s->slot_req[i]) { slot = i; break; }
    q->slot = slot;
    s->slot_req[slot] = q;
    pcg::ServeSlot& hs = s->h_slots[slot];
    hs.op = q->op32;
    hs.u = q->u; hs.r = q->r; hs.z = q->z; hs.p = q->p; hs.q = q->q;
    hs.st = s->d_states + 2 * slot;
    hs.partials = q->partials;
    hs.counter = q->counter;
    hs.gx = q->gx;
    hs.nch = q->nch;
    hs.rows = q->rows;
    hs.colmode = q->colmode;
    hs.nprec = q->nprec;
    hs.nspmv = q->nspmv;
    hs.tmaps = q->tmaps;
    hs.prec_tma = q->prec_tma;
    hs.ptab = (tab && q->prec_tma) ? ptab : nullptr;
    SRV_CK(s, cudaMemcpyAsync(s->d_slots + slot, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
    pcg::k_init_state<<<1, 32, 0, st>>>(s->d_states + 2 * slot, 2, 0.0, 0, nullptr);
    s->launches += 1;
    s->used += q->bytes;
    s->active_unknowns += (long long)vol;
    q->phase = RQ_MEASURE;
    q->t_admit = now_ms();
    q->b.clear();
    q->b.shrink_to_fit();
    return PCG_OK;
}

int retire(pcg_server_t s, ServeReq* q) {
    q->x.resize((size_t)q->grid.n_x * q->grid.n_y * q->grid.n_z);
    SRV_CK(s, cudaMemcpyAsync(q->x.data(), q->xd, q->x.size() * 8, cudaMemcpyDeviceToHost, s->stream));
    SRV_CK(s, cudaFreeAsync(q->dmem, s->stream));
    SRV_CK(s, cudaStreamSynchronize(s->stream));
    s->used -= q->bytes;
    s->active_unknowns -= (long long)q->grid.n_x * q->grid.n_y * q->grid.n_z;
    q->dmem = nullptr;
    s->slot_req[q->slot] = nullptr;
    q->slot = -1;
    q->phase = RQ_DONE;
    q->t_done = now_ms();
    s->retired += 1;
    return PCG_OK;
}

// FP64 refinement step of every request in the measure phase: true residual,
// then (per request, on the host) retire, or coarse correction + emit the
// inner right-hand side + reset the inner state.
int measure_and_decide(pcg_server_t s) {
    std::vector<ServeReq*> ms;
    for (ServeReq* q : s->slot_req)
        if (q && q->phase == RQ_MEASURE) ms.push_back(q);
    if (ms.empty()) return PCG_OK;
    cudaStream_t st = s->stream;
    for (ServeReq* q : ms) {
        SolveState* so = s->d_states + 2 * q->slot + 1;
        pcg::k_residual<float><<<dim3(q->gx, q->gy, 1), dim3(BX, BY, 1), 0, st>>>(
            q->op64, q->bd, q->xd, nullptr, (float*)nullptr, so, q->partials, q->counter, q->ntiles, 2);
    }
    s->launches += (long long)ms.size();
    SRV_CK(s, cudaGetLastError());
    SRV_CK(s, cudaMemcpyAsync(s->h_states, s->d_states, sizeof(SolveState) * 2 * s->max_slots,
                              cudaMemcpyDeviceToHost, st));
    SRV_CK(s, cudaStreamSynchronize(st));
    for (ServeReq* q : ms) {
        const SolveState& o = s->h_states[2 * q->slot + 1];
        q->bb = o.bnorm2;
        q->last_rr = o.rr;
        bool stop = false;
        if (q->bb == 0.0) {
            q->status = PCG_OK;
            q->last_rr = 0.0;
            stop = true;
        } else {
            const double rel = std::sqrt(o.rr / q->bb);
            q->floor_rel = std::sqrt(o.floor2 / q->bb);
            q->hist.push_back(rel);
            if (s->trace)
                std::fprintf(stderr, "[serve] req %llu slot %d sweep %d relres_true %.3e floor %.3e inner_its %d\n",
                             (unsigned long long)q->id, q->slot, q->sweeps, rel, q->floor_rel, q->inner_its);
            if (!std::isfinite(rel)) { q->status = PCG_BREAKDOWN; stop = true; }
            else if (rel < q->tol) { q->status = PCG_OK; stop = true; }
            else if (rel <= 2.0 * q->floor_rel) { q->status = PCG_OK; q->stag = 1; stop = true; }
            else if (q->hist.size() >= 4) {
                const double best_now = *std::min_element(q->hist.begin(), q->hist.end());
                const double best_before = *std::min_element(q->hist.begin(), q->hist.end() - 3);
                if (best_now > 0.5 * best_before) { q->status = PCG_OK; q->stag = 1; stop = true; }
            }
            if (!stop && q->sweeps >= s->max_outer) { q->status = PCG_NOT_CONVERGED; stop = true; }
        }
        if (q->status == PCG_BREAKDOWN) stop = true;
        if (stop) {
            int rc = retire(s, q);
            if (rc) return rc;
            s->items_dirty = true;
            continue;
        }
        SolveState* si = s->d_states + 2 * q->slot;
        SolveState* so = si + 1;
        const size_t vol = (size_t)q->op32.vol;
        pcg::k_coarse<<<1, 32, 0, st>>>(so, 1, q->total_mass);
        pcg::k_residual<float><<<dim3(q->gx, q->gy, 1), dim3(BX, BY, 1), 0, st>>>(
            q->op64, q->bd, q->xd, nullptr, q->r, so, q->partials, q->counter, q->ntiles, 3);
        pcg::k_init_state<<<1, 32, 0, st>>>(si, 1, 0.0, s->inner_maxit, nullptr);
        pcg::k_inner_thresholds<<<1, 32, 0, st>>>(si, so, 1, s->inner_tol * s->inner_tol);
        SRV_CK(s, cudaMemsetAsync(q->u, 0, vol * 4, st));
        SRV_CK(s, cudaMemsetAsync(q->p, 0, vol * 4, st));
        SRV_CK(s, cudaMemsetAsync(q->q, 0, vol * 4, st));
        SRV_CK(s, cudaGetLastError());
        s->launches += 4;
        q->phase = RQ_INNER;
        s->items_dirty = true;
    }
    return PCG_OK;
}

int rebuild_items(pcg_server_t s) {
    long long na = 0, nb = 0;
    for (ServeReq* q : s->slot_req)
        if (q && q->phase == RQ_INNER) { na += q->nprec; nb += q->nspmv; }
    if (na > s->items_cap || nb > s->items_cap) return sfail(s, PCG_ERR_OOM, "work list capacity exceeded");
    int2* ha = s->h_items;
    int2* hb = s->h_items + s->items_cap;
    int ka = 0, kb = 0;
    for (ServeReq* q : s->slot_req) {
        if (!q || q->phase != RQ_INNER) continue;
        for (int t = 0; t < q->nprec; ++t) ha[ka++] = make_int2(q->slot, t);
        for (int t = 0; t < q->nspmv; ++t) hb[kb++] = make_int2(q->slot, t);
    }
    s->h_nitems[0] = (int)na;
    s->h_nitems[1] = (int)nb;
    for (int i = 0; i < s->max_slots; ++i) s->h_inner[i] = (s->slot_req[i] && s->slot_req[i]->phase == RQ_INNER) ? 1 : 0;
    SRV_CK(s, cudaMemcpyAsync(s->d_inner, s->h_inner, sizeof(int) * (size_t)s->max_slots, cudaMemcpyHostToDevice,
                              s->stream));
    SRV_CK(s, cudaMemcpyAsync(s->d_items, ha, sizeof(int2) * (size_t)std::max<long long>(na, 1),
                              cudaMemcpyHostToDevice, s->stream));
    SRV_CK(s, cudaMemcpyAsync(s->d_items + s->items_cap, hb, sizeof(int2) * (size_t)std::max<long long>(nb, 1),
                              cudaMemcpyHostToDevice, s->stream));
    SRV_CK(s, cudaMemcpyAsync(s->d_nitems, s->h_nitems, 2 * sizeof(int), cudaMemcpyHostToDevice, s->stream));
    s->items_dirty = false;
    return PCG_OK;
}

int capture_epochs(pcg_server_t s) {
    cudaGraph_t g = nullptr;
    SRV_CK(s, cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
    // every launch takes its items in arrival order from a counter of its own
    SRV_CK(s, cudaMemsetAsync(s->d_fetch, 0, 2 * sizeof(unsigned) * (size_t)s->epochs_per_launch, s->cap_stream));
    for (int e = 0; e < s->epochs_per_launch; ++e) {
        pcg::k_serve_prec<2><<<s->blocks_prec, dim3(BX, 8, 1), pcg::SERVE_PREC_SMEM, s->cap_stream>>>(
            s->d_slots, s->d_items, s->d_nitems, s->d_fetch + 2 * e);
        pcg::k_serve_scalars<0><<<s->max_slots, 256, 0, s->cap_stream>>>(s->d_slots, s->d_inner);
        pcg::k_serve_spmv<<<s->blocks_spmv, dim3(BX, pcg::SERVE_BY, 1), pcg::SERVE_SPMV_SMEM, s->cap_stream>>>(
            s->d_slots, s->d_items + s->items_cap, s->d_nitems + 1, s->d_fetch + 2 * e + 1);
        pcg::k_serve_scalars<1><<<s->max_slots, 256, 0, s->cap_stream>>>(s->d_slots, s->d_inner);
    }
    cudaError_t e = cudaStreamEndCapture(s->cap_stream, &g);
    if (e != cudaSuccess) return sfail(s, PCG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return sfail(s, PCG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return PCG_OK;
}

}  // namespace

#include "serve_mg.cuh"

extern "C" {

int pcg_server_create(size_t budget_bytes, int max_slots, const pcg_opts_t* opts, pcg_server_t* out) {
    if (!out) return sfail(nullptr, PCG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (budget_bytes == 0 || max_slots < 1 || max_slots > 4096)
        return sfail(nullptr, PCG_ERR_INVALID_ARG, "budget_bytes must be > 0 and 1 <= max_slots <= 4096");
    pcg_server* s = new (std::nothrow) pcg_server();
    if (!s) return sfail(nullptr, PCG_ERR_OOM, "host allocation failed");
    s->budget = budget_bytes;
    s->max_slots = max_slots;
    if (const char* tr = std::getenv("PCG_TRACE")) s->trace = std::atoi(tr);
    if (opts) {
        if (opts->inner_tol > 0) s->inner_tol = opts->inner_tol;
        if (opts->inner_maxit > 0) s->inner_maxit = opts->inner_maxit;
        if (opts->max_outer > 0) s->max_outer = opts->max_outer;
        if (opts->passes_per_launch > 0) s->epochs_per_launch = opts->passes_per_launch;
        s->stream = (cudaStream_t)opts->stream;
    }
    auto bail = [&](int rc) {
        g_create_error = s->err;
        g_null_error = nullptr;
        pcg_server_destroy(s);
        return rc;
    };
    cudaError_t e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) { s->err = cudaGetErrorString(e); return bail(PCG_ERR_CUDA); }
    s->device = dev;
    const int pc = opts ? opts->preconditioner : PCG_PREC_LINE;
    if (pc != PCG_PREC_LINE && pc != PCG_PREC_MULTIGRID_F32) {
        s->err = "served solves take the line preconditioner or PCG_PREC_MULTIGRID_F32";
        return bail(PCG_ERR_INVALID_ARG);
    }
    if (pc == PCG_PREC_MULTIGRID_F32) {
        // multigrid mode: up to 16 requests solved at once, one worker thread and stream each
        s->mode = 1;
        const int nw = std::min(max_slots, 16);
        try {
            for (int i = 0; i < nw; ++i) s->workers.emplace_back(mg_worker, s);
        } catch (...) {
            s->err = "could not start the worker threads";
            return bail(PCG_ERR_OOM);
        }
        *out = s;
        return PCG_OK;
    }
    s->slot_req.assign(max_slots, nullptr);
    s->h_slots.assign(max_slots, pcg::ServeSlot{});
    s->items_cap = 1 << 21;
    if ((e = cudaDeviceGetDefaultMemPool(&s->pool, dev)) != cudaSuccess) { s->err = cudaGetErrorString(e); return bail(PCG_ERR_CUDA); }
    if ((e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        s->err = cudaGetErrorString(e);
        return bail(PCG_ERR_CUDA);
    }
    struct { void** p; size_t b; } dev_allocs[] = {
        {(void**)&s->d_slots, sizeof(pcg::ServeSlot) * max_slots},
        {(void**)&s->d_states, sizeof(SolveState) * 2 * max_slots},
        {(void**)&s->d_items, 2 * sizeof(int2) * (size_t)s->items_cap},
        {(void**)&s->d_nitems, 2 * sizeof(int)},
        {(void**)&s->d_one, sizeof(int)},
        {(void**)&s->d_inner, sizeof(int) * (size_t)max_slots},
        {(void**)&s->d_fetch, 2 * sizeof(unsigned) * (size_t)std::max(s->epochs_per_launch, 1)},
    };
    for (auto& a : dev_allocs)
        if ((e = cudaMalloc(a.p, a.b)) != cudaSuccess) { *a.p = nullptr; s->err = "cudaMalloc failed"; return bail(PCG_ERR_OOM); }
    if ((e = cudaMallocHost((void**)&s->h_states, sizeof(SolveState) * 2 * max_slots)) != cudaSuccess ||
        (e = cudaMallocHost((void**)&s->h_items, 2 * sizeof(int2) * (size_t)s->items_cap)) != cudaSuccess ||
        (e = cudaMallocHost((void**)&s->h_nitems, 2 * sizeof(int))) != cudaSuccess ||
        (e = cudaMallocHost((void**)&s->h_inner, sizeof(int) * (size_t)max_slots)) != cudaSuccess) {
        s->err = "cudaMallocHost failed";
        return bail(PCG_ERR_OOM);
    }
    const int one = 1;
    if ((e = cudaMemcpy(s->d_one, &one, sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(s->d_nitems, 0, 2 * sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(s->d_inner, 0, sizeof(int) * (size_t)max_slots)) != cudaSuccess ||
        (e = cudaMemset(s->d_slots, 0, sizeof(pcg::ServeSlot) * max_slots)) != cudaSuccess) {
        s->err = cudaGetErrorString(e);
        return bail(PCG_ERR_CUDA);
    }
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // persistent grids: as many blocks as are resident on every SM at once
    if ((e = cudaFuncSetAttribute(pcg::k_serve_spmv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)pcg::SERVE_SPMV_SMEM)) != cudaSuccess) {
        s->err = cudaGetErrorString(e);
        return bail(PCG_ERR_CUDA);
    }
    if ((e = cudaFuncSetAttribute(pcg::k_serve_prec<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)pcg::SERVE_PREC_SMEM)) != cudaSuccess) {
        s->err = cudaGetErrorString(e);
        return bail(PCG_ERR_CUDA);
    }
    int occ_a = 0, occ_b = 0;
    const cudaError_t eo =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_a, pcg::k_serve_prec<2>, BX * 8, pcg::SERVE_PREC_SMEM);
    if (eo != cudaSuccess || occ_a < 1) occ_a = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, pcg::k_serve_spmv, BX * pcg::SERVE_BY,
                                                      pcg::SERVE_SPMV_SMEM) != cudaSuccess || occ_b < 1)
        occ_b = 1;
    s->blocks_prec = sms * occ_a;
    s->blocks_spmv = sms * occ_b;
    *out = s;
    return PCG_OK;
}

int pcg_serve_submit(pcg_server_t s, const pcg_grid_t* grid, const pcg_coeffs_t* coeffs, const double* b_host,
                     double tol, uint64_t* req_id) {
    if (!s) return sfail(nullptr, PCG_ERR_INVALID_ARG, "server is NULL");
    if (!grid || !coeffs || !b_host || !req_id) return sfail(s, PCG_ERR_INVALID_ARG, "grid, coeffs, b and req_id are required");
    if (grid->n_x < 1 || grid->n_y < 1 || grid->n_z < 1) return sfail(s, PCG_ERR_INVALID_ARG, "n_x, n_y, n_z must be >= 1");
    if (grid->nrhs != 1) return sfail(s, PCG_ERR_INVALID_ARG, "served requests have one right-hand side");
    if (!grid->z_iface || !coeffs->beta_iface) return sfail(s, PCG_ERR_INVALID_ARG, "z_iface and beta_iface are required");
    if (!(tol >= 0.0)) return sfail(s, PCG_ERR_INVALID_ARG, "tol must be >= 0");
    // validate the tables now so that a bad request fails at submission
    {
        HostTables t;
        std::string err;
        double tm = 0.0;
        const int rc = build_tables_core(grid, coeffs, t, err, tm);
        if (rc) return sfail(s, rc, err);
    }
    const int cls_mode = serve_cls_mode(*grid, coeffs->alpha_e || coeffs->alpha_n);
    const size_t need = s->mode == 1 ? mg_request_bytes(*grid) : request_bytes(*grid, cls_mode);
    if (need > s->budget) return sfail(s, PCG_ERR_OOM, "request needs more device memory than the server's budget");
    ServeReq* q = new (std::nothrow) ServeReq();
    if (!q) return sfail(s, PCG_ERR_OOM, "host allocation failed");
    q->grid = *grid;
    const size_t nz = grid->n_z, nxy = (size_t)grid->n_x * grid->n_y;
    q->z_iface.assign(grid->z_iface, grid->z_iface + nz + 1);
    q->beta.assign(coeffs->beta_iface, coeffs->beta_iface + nz + 1);
    if (coeffs->alpha_e) q->alpha_e.assign(coeffs->alpha_e, coeffs->alpha_e + nxy);
    if (coeffs->alpha_n) q->alpha_n.assign(coeffs->alpha_n, coeffs->alpha_n + nxy);
    q->lambda2 = coeffs->lambda2;
    q->b.assign(b_host, b_host + nxy * nz);
    q->tol = tol;
    q->t_submit = now_ms();
    if (s->mode == 1) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            q->id = s->next_id++;
            s->pending.push_back(q);
            s->reqs[q->id] = q;
        }
        s->cv_work.notify_all();
        *req_id = q->id;
        return PCG_OK;
    }
    q->id = s->next_id++;
    s->pending.push_back(q);
    s->reqs[q->id] = q;
    *req_id = q->id;
    return PCG_OK;
}

int pcg_serve_step(pcg_server_t s, int max_epochs, int* n_active, int* n_pending) {
    if (!s) return sfail(nullptr, PCG_ERR_INVALID_ARG, "server is NULL");
    if (s->mode == 1) {
        // the workers advance on their own: wait (at most a millisecond) for one to finish a request
        std::unique_lock<std::mutex> lk(s->mu);
        const long long before = s->retired;
        s->cv_done.wait_for(lk, std::chrono::milliseconds(1), [&] { return s->retired != before; });
        if (n_active) *n_active = s->busy;
        if (n_pending) *n_pending = (int)s->pending.size();
        return PCG_OK;
    }
    if (!s->graph) {
        int rc = capture_epochs(s);
        if (rc) return rc;
    }
    int done_epochs = 0;
    for (;;) {
        // admission: FIFO while a slot and the budget allow
        int admitted = 0;
        while (!s->pending.empty()) {
            ServeReq* q = s->pending.front();
            bool free_slot = false;
            for (ServeReq* r : s->slot_req) if (!r) { free_slot = true; break; }
            const int cls_mode = serve_cls_mode(q->grid, !q->alpha_e.empty() || !q->alpha_n.empty());
            if (!free_slot || s->used + request_bytes(q->grid, cls_mode) > s->budget) break;
            s->pending.pop_front();
            int rc = admit(s, q);
            if (rc) return rc;
            ++admitted;
        }
        int rc = measure_and_decide(s);
        if (rc) return rc;
        int n_inner = 0;
        for (ServeReq* q : s->slot_req) if (q && q->phase == RQ_INNER) ++n_inner;
        if (n_inner == 0) {
            bool any_active = false;
            for (ServeReq* q : s->slot_req) if (q) any_active = true;
            if (s->pending.empty() || (!admitted && any_active)) break;
            if (!admitted && !any_active) continue;   // everything retired: the queue head fits now
            continue;                                 // retirements freed room: admit more
        }
        if (done_epochs >= max_epochs) break;
        if (s->items_dirty && (rc = rebuild_items(s)) != PCG_OK) return rc;
        SRV_CK(s, cudaGraphLaunch(s->graph, s->stream));
        s->launches += 4LL * s->epochs_per_launch;   // two sweeps and their scalar steps per epoch
        s->epochs += s->epochs_per_launch;
        done_epochs += s->epochs_per_launch;
        SRV_CK(s, cudaMemcpyAsync(s->h_states, s->d_states, sizeof(SolveState) * 2 * s->max_slots,
                                  cudaMemcpyDeviceToHost, s->stream));
        SRV_CK(s, cudaStreamSynchronize(s->stream));
        for (ServeReq* q : s->slot_req) {
            if (!q || q->phase != RQ_INNER) continue;
            const SolveState& si = s->h_states[2 * q->slot];
            if (!si.done) continue;
            q->sweeps += 1;
            q->inner_its += std::max(0, si.pass - 1);
            if (si.status == PCG_BREAKDOWN || si.status == PCG_TIMEOUT) {
                q->status = si.status;
                rc = retire(s, q);
                if (rc) return rc;
                s->items_dirty = true;
                continue;
            }
            pcg::k_refine_update<<<dim3(q->gx, q->gy, 1), dim3(BX, BY, 1), 0, s->stream>>>(
                q->grid.n_x, q->grid.n_y, q->grid.n_z, q->op64.plane, q->op64.vol, q->xd, q->u, q->p,
                s->d_states + 2 * q->slot, s->d_states + 2 * q->slot + 1, s->d_one);
            s->launches += 1;
            q->phase = RQ_MEASURE;
            s->items_dirty = true;
        }
        SRV_CK(s, cudaGetLastError());
    }
    int act = 0;
    for (ServeReq* q : s->slot_req) if (q) ++act;
    if (n_active) *n_active = act;
    if (n_pending) *n_pending = (int)s->pending.size();
    return PCG_OK;
}

int pcg_serve_poll(pcg_server_t s, uint64_t req_id, double* x_host, pcg_stats_t* stats) {
    if (!s) return sfail(nullptr, PCG_ERR_INVALID_ARG, "server is NULL");
    if (s->mode == 1) {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->reqs.find(req_id);
        if (it == s->reqs.end()) return sfail(s, PCG_ERR_INVALID_ARG, "unknown request id");
        ServeReq* q = it->second;
        if (q->phase != RQ_DONE) return PCG_PENDING;
        s->reqs.erase(it);
        lk.unlock();
        if (x_host && !q->x.empty()) std::memcpy(x_host, q->x.data(), q->x.size() * sizeof(double));
        if (stats) {
            *stats = q->mg_stats;
            stats->elapsed_ms = q->t_done - q->t_submit;
        }
        delete q;
        return PCG_OK;
    }
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return sfail(s, PCG_ERR_INVALID_ARG, "unknown request id");
    ServeReq* q = it->second;
    if (q->phase != RQ_DONE) return PCG_PENDING;
    if (x_host) std::memcpy(x_host, q->x.data(), q->x.size() * sizeof(double));
    if (stats) {
        pcg_stats_t o{};
        o.status = q->status;
        o.iterations = q->inner_its;
        o.outer_sweeps = q->sweeps;
        o.stagnated = q->stag;
        o.relres_true = q->bb > 0 ? std::sqrt(q->last_rr / q->bb) : 0.0;
        o.relres_recursive = o.relres_true;
        o.relres_floor = q->floor_rel;
        o.elapsed_ms = q->t_done - q->t_submit;
        *stats = o;
    }
    s->reqs.erase(it);
    delete q;
    return PCG_OK;
}

int pcg_serve_info(pcg_server_t s, int* n_active, int* n_pending, size_t* used_bytes, long long* epochs) {
    if (!s) return sfail(nullptr, PCG_ERR_INVALID_ARG, "server is NULL");
    if (s->mode == 1) {
        std::lock_guard<std::mutex> lk(s->mu);
        if (n_active) *n_active = s->busy;
        if (n_pending) *n_pending = (int)s->pending.size();
        if (used_bytes) *used_bytes = s->used;
        if (epochs) *epochs = 0;
        return PCG_OK;
    }
    int act = 0;
    for (ServeReq* q : s->slot_req) if (q) ++act;
    if (n_active) *n_active = act;
    if (n_pending) *n_pending = (int)s->pending.size();
    if (used_bytes) *used_bytes = s->used;
    if (epochs) *epochs = s->epochs;
    return PCG_OK;
}

const char* pcg_server_last_error(pcg_server_t s) { return s ? s->err.c_str() : g_create_error.c_str(); }

void pcg_server_destroy(pcg_server_t s) {
    if (!s) return;
    if (s->mode == 1) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stopping = true;
        }
        s->cv_work.notify_all();
        for (auto& t : s->workers) t.join();   // a worker finishes the request it is solving first
        for (auto& kv : s->reqs) delete kv.second;
        delete s;
        return;
    }
    cudaStreamSynchronize(s->stream);
    for (auto& kv : s->reqs) {
        ServeReq* q = kv.second;
        if (q->dmem) cudaFreeAsync(q->dmem, s->stream);
        delete q;
    }
    cudaStreamSynchronize(s->stream);
    if (s->graph) cudaGraphExecDestroy(s->graph);
    for (void* p : {(void*)s->d_slots, (void*)s->d_states, (void*)s->d_items, (void*)s->d_nitems, (void*)s->d_one,
                    (void*)s->d_inner, (void*)s->d_fetch})
        if (p) cudaFree(p);
    for (void* p : {(void*)s->h_states, (void*)s->h_items, (void*)s->h_nitems, (void*)s->h_inner})
        if (p) cudaFreeHost(p);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    delete s;
}

}  // extern "C"
