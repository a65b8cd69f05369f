// Served solves with the multigrid preconditioner (a server created with
// opts->preconditioner == PCG_PREC_MULTIGRID_F32).
//
// Each request is solved by FP64 CG (Algorithm 1) preconditioned by one FP32
// V-cycle of the geometric multigrid, the solver the paper names as its next
// step: about twenty iterations where the line-preconditioned mixed form needs
// a thousand or more.  A pool of worker threads, each with a stream of its own,
// takes the queued requests in arrival order while the device-byte budget
// allows, builds each one's solver (tables, factors, coarse levels) in a
// handle of its own, solves it (restarting CG from x until the true residual
// meets the tolerance or the FP64 rounding floor, as the mixed form's
// refinement does), copies x out and frees the handle.  Requests
// that arrive while others are being solved are admitted as soon as a worker
// and the budget free up, and the work of the requests in flight overlaps on
// the device (their kernels run from different streams).  A request's
// arithmetic is that of pcg_solve on its own handle, so its result does not
// depend on the other requests.
#include <condition_variable>
#include <mutex>
#include <thread>

namespace {

// Device bytes a request holds while it is solved: FP64 workspace, host-copy
// staging, the V-cycle's FP32 vectors on every level and the tables (an upper
// bound of 96 bytes per unknown).
size_t mg_request_bytes(const pcg_grid_t& g) {
    return (size_t)g.n_x * g.n_y * g.n_z * 96 + (size_t(1) << 20);
}

bool mg_can_admit(const pcg_server* s) {
    if (s->pending.empty()) return false;
    return s->busy == 0 || s->used + mg_request_bytes(s->pending.front()->grid) <= s->budget;
}

// One request, on the worker's stream: its own handle, pcg_solve_host, free.
void mg_solve_one(ServeReq* q, cudaStream_t st) {
    pcg_grid_t g = q->grid;
    g.z_iface = q->z_iface.data();
    g.nrhs = 1;
    pcg_coeffs_t c{};
    c.beta_iface = q->beta.data();
    c.alpha_e = q->alpha_e.empty() ? nullptr : q->alpha_e.data();
    c.alpha_n = q->alpha_n.empty() ? nullptr : q->alpha_n.data();
    c.lambda2 = q->lambda2;
    pcg_opts_t o{};
    o.precision = PCG_FP64;
    o.preconditioner = PCG_PREC_MULTIGRID_F32;
    // 16 passes per graph launch, not the 4 a lone multigrid solve takes:
    // with up to 16 workers polling, fewer and longer launches measured
    // faster, and other requests' work covers a solve's trailing early exits
    o.passes_per_launch = 16;
    o.stream = (void*)st;
    pcg_t h = nullptr;
    pcg_stats_t res{};
    int rc = pcg_create(&g, &c, &o, &h);
    if (rc == PCG_OK) {
        // CG stops on its updated residual, which drifts from the true one; as
        // the mixed form's refinement does, the solve is restarted from x (a
        // fresh FP64 residual) until the true residual is below tol or within
        // twice the FP64 rounding floor of x, at most four solves in all
        q->x.assign((size_t)g.n_x * g.n_y * g.n_z, 0.0);
        int its = 0, solves = 0;
        for (;;) {
            rc = pcg_solve_host(h, q->b.data(), q->x.data(), q->tol, 100000, &res);
            its += res.iterations;
            solves += 1;
            if (rc != PCG_OK || res.status != PCG_OK) break;
            if (res.relres_true < q->tol || res.relres_true <= 2.0 * res.relres_floor) break;
            if (solves == 4) {
                res.stagnated = 1;
                break;
            }
        }
        if (rc != PCG_OK && rc != PCG_NOT_CONVERGED && rc != PCG_BREAKDOWN) res.status = rc;
        res.iterations = its;
        res.outer_sweeps = solves;
        pcg_destroy(h);
    } else {
        res.status = rc;
    }
    q->status = res.status;
    q->mg_stats = res;
    q->b.clear();
    q->b.shrink_to_fit();
}

void mg_worker(pcg_server_t s) {
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    for (;;) {
        ServeReq* q = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stopping || (st && mg_can_admit(s)); });
            if (s->stopping) break;
            q = s->pending.front();
            s->pending.pop_front();
            q->bytes = mg_request_bytes(q->grid);
            s->used += q->bytes;
            s->busy += 1;
            q->phase = RQ_INNER;
            q->t_admit = now_ms();
        }
        mg_solve_one(q, st);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->used -= q->bytes;
            s->busy -= 1;
            s->retired += 1;
            q->t_done = now_ms();
            q->phase = RQ_DONE;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    if (st) cudaStreamDestroy(st);
}

}  // namespace
