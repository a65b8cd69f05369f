// Device kernels of the served batch (pcg_server_*): persistent sweeps over
// work lists of (request slot, item) of all admitted requests.
#pragma once
#include "kernels.cuh"

namespace pcg {

// ---------------------------------------------------------------------------
// Served batch: persistent sweeps over work lists of (request slot, item).
//
// Every admitted request owns a slot with its own tables, vectors, partials,
// and scalar state.  One launch of each kernel walks all items of all
// requests in the inner phase, so many small solves fill the GPU together;
// every item writes its block's partial sums, and k_serve_scalars then forms
// each request's scalars from its own partials in a fixed order, so a
// request's arithmetic does not depend on which other requests share the
// launch.
//   k_serve_prec: 256-thread blocks; an item is `rows` rows of 32 columns,
//     each column split into nch chunks of 16 levels (one warp per chunk,
//     prec_chunked_body), its r and q staged in shared memory by bulk tensor
//     copies of the request's own maps, two items ahead (as k_sweep_prec_tma);
//     columns of more than 128 levels take one thread per column (8 rows per
//     item, prec_column), and requests without maps read r and q directly.
//   k_serve_spmv: 128-thread blocks; an item is a 32 x 4-column tile of one
//     16-level chunk, staged in shared memory by bulk tensor copies (tensor
//     maps of the request in device memory) or, when the request's rows are
//     not 16-byte multiples, by the threads; then spmv_tile_compute.
// ---------------------------------------------------------------------------
constexpr int SERVE_LZ = 16, SERVE_BY = 4;

struct ServeSlot {
    OpView<float> op;           // FP32 tables of the request
    float *u, *r, *z, *p, *q;   // inner FP32 vectors
    SolveState* st;             // inner state
    double* partials;           // [max(nprec, nspmv)][4]
    unsigned* counter;
    int gx;                     // tiles of 32 columns per row
    int nch;                    // chunks of 16 levels per column
    int rows;                   // preconditioner: rows per item
    int colmode;                // preconditioner: 1 = one thread per column (n_z > 128)
    int nprec;                  // preconditioner items
    int nspmv;                  // SpMV items: gx * ceil(n_y / 8) * nch
    const CUtensorMap* tmaps;   // [4] u, p, q, z (boxes as k_sweep_spmv_tma), then [2] r, q (box 32 x rows x
                                // 16 nch), or null
    int prec_tma;               // 1: the preconditioner items are staged through tmaps[4], tmaps[5]
    const float* ptab;          // [5][n_z]: 1/D, E, e, C, Q of PrecTab (one factor set, items of 1, 2 or 4
                                // rows of whole 16-level chunks), or null
};

// The carry tables of a request with one factor set, built once at admission
// (one block of 256 threads) by the routine the one-request sweep uses.
__global__ __launch_bounds__(256) void k_build_prec_tab(OpView<float> op, float* __restrict__ dst) {
    __shared__ PrecTab<SERVE_LZ> tb;
    const int tid = threadIdx.x, nz = op.nz;
    prec_tab_build<SERVE_LZ>(op, tb, tid, 256);
    for (int k = tid; k < nz; k += 256) {
        dst[k] = tb.g[k];
        dst[nz + k] = tb.E[k];
        dst[2 * nz + k] = tb.e[k];
        dst[3 * nz + k] = tb.C[k];
        dst[4 * nz + k] = tb.Q[k];
    }
}

constexpr int SERVE_PVN = 8 * SERVE_LZ * 32;   // floats of one vector in one stage (rows x nch <= 8)
constexpr size_t SERVE_PREC_SMEM = 4 * (size_t)SERVE_PVN * 4 + 16 + 128;   // 2 stages x (r, q), 2 mbarriers

__device__ __forceinline__ void tmap_acquire(const CUtensorMap* m) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" :: "l"(reinterpret_cast<uint64_t>(m)) : "memory");
}

// The served preconditioner's less common item kinds, kept out of line so
// that their register needs do not weigh on the tabulated path: columns of
// more than 128 levels (one thread per column) and items without the carry
// tables (staged, or read directly from r and q).
__device__ __noinline__ void serve_prec_column(const ServeSlot& s, int bx, int jb, int lane, int w, float alpha,
                                               Acc<float> (&acc)[2]) {
    const Col<float> col = make_col(s.op, bx * 32 + lane, jb * 8 + w);
    if (col.valid) prec_column<float>(s.op, col, s.r + col.c, s.q + col.c, s.z + col.c, alpha, acc[0], acc[1]);
}

__device__ __noinline__ void serve_prec_generic(const ServeSlot& s, const Col<float>& col, int lane, int ch, int row,
                                                float alpha, Acc<float> (&acc)[2], float (*sh_y)[32],
                                                float (*sh_c)[32], float (*sh_z)[32], float (*sh_d)[32],
                                                const float* rs) {
    if (rs)
        prec_chunked_body<float, SERVE_LZ>(s.op, col, lane, ch, s.nch, row * s.nch, s.r, s.q, s.z, alpha, acc, sh_y,
                                           sh_c, sh_z, sh_d, rs, rs + SERVE_PVN, s.rows * 32);
    else
        prec_chunked_body<float, SERVE_LZ>(s.op, col, lane, ch, s.nch, row * s.nch, s.r, s.q, s.z, alpha, acc, sh_y,
                                           sh_c, sh_z, sh_d);
}

// The tabulated chunked solve of one staged item, one function per item
// height, each with its own register allocation.
template <int R>
__device__ __noinline__ void serve_prec_tab(const ServeSlot& s, const PrecTab<SERVE_LZ>& tb, const Col<float>& col,
                                            int lane, int ch, int row, float alpha, Acc<float> (&acc)[2],
                                            float (*sh_y)[32], float (*sh_c)[32], float (*sh_z)[32],
                                            float (*sh_d)[32], const float* rs) {
    prec_tab_body<SERVE_LZ, R, true>(s.op, tb, col, lane, ch, s.nch, row * s.nch, s.r, s.z, alpha, acc, sh_y, sh_c,
                                     sh_z, sh_d, rs, rs + SERVE_PVN);
}

// Items are taken in arrival order from `fetch` (zeroed before the launch):
// thread 0 draws an item when it refills a stage, so a block's stages hold its
// items in the order drawn, and once one of them is past the end of the list
// every later draw of the block is too.
template <int MINB>
__global__ __launch_bounds__(256, MINB) void k_serve_prec(const ServeSlot* __restrict__ slots,
                                                         const int2* __restrict__ items,
                                                         const int* __restrict__ n_items,
                                                         unsigned* __restrict__ fetch) {
    __shared__ float sh_y[MAXW][32], sh_c[MAXW][32], sh_z[MAXW][32], sh_d[MAXW][32];
    __shared__ int staged[2];       // stage g holds the bulk copies of its item (1) or nothing (0)
    __shared__ int stage_item[2];   // the item drawn for stage g (n or more: none)
    __shared__ PrecTab<SERVE_LZ> tb;   // the carry tables of the item's request (ptab)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* sbase = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint64_t* bars = reinterpret_cast<uint64_t*>(sbase + 4 * SERVE_PVN);
    const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane;
    const uint32_t bar0 = smem_u32(bars), bar1 = smem_u32(bars + 1);
    const int n = *n_items;
    int last_slot = -1;   // thread 0: the slot whose maps it acquired last
    bool ok = true;       // false once a copy failed to land in time: no more copies are started
    // thread 0: draw the next item for stage g and start its copies if its
    // request is staged and running
    auto issue = [&](int g) {
        const int it = (int)atomicAdd(fetch, 1u);
        stage_item[g] = it;
        int go = 0;
        if (ok && it < n) {
            const int2 wk = items[it];
            const ServeSlot& s = slots[wk.x];
            if (s.prec_tma && !s.colmode && !s.st->done) {
                if (wk.x != last_slot) {
                    tmap_acquire(s.tmaps + 4);
                    tmap_acquire(s.tmaps + 5);
                    last_slot = wk.x;
                }
                const uint32_t bar = g ? bar1 : bar0;
                float* rs = sbase + g * 2 * SERVE_PVN;
                const int bx = wk.y % s.gx, jb = wk.y / s.gx;
                // earlier items read the stage through the generic proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect(bar, 2u * 32u * (uint32_t)s.rows * (uint32_t)(s.nch * SERVE_LZ) * 4u);
                tma_load_3d(smem_u32(rs), s.tmaps + 4, bx * 32, jb * s.rows, 0, bar);
                tma_load_3d(smem_u32(rs + SERVE_PVN), s.tmaps + 5, bx * 32, jb * s.rows, 0, bar);
                go = 1;
            }
        }
        staged[g] = go;
    };
    if (tid == 0) {
        mbar_init(bar0);
        mbar_init(bar1);
        issue(0);
        issue(1);
    }
    __syncthreads();
    uint32_t par0 = 0, par1 = 0;
    bool pend0 = false, pend1 = false;   // a copy into the stage that has not been seen to land
    for (int k = 0;; ++k) {
        const int g = k & 1;
        // stage_item[g] and staged[g] were written before the barriers of the previous item
        const int it = stage_item[g];
        if (it >= n) break;
        const int2 wk = items[it];
        const ServeSlot& s = slots[wk.x];
        SolveState* st = s.st;
        const bool was_staged = staged[g] != 0;
        bool landed = true;
        if (was_staged) {
            const bool l = mbar_wait(g ? bar1 : bar0, g ? par1 : par0, 1 << 22);
            landed = __syncthreads_and(l ? 1 : 0) != 0;
            if (landed) {
                if (g) par1 ^= 1u; else par0 ^= 1u;
            } else {
                if (tid == 0) atomicExch(&st->status, 6);   // PCG_TIMEOUT: this item is not computed
                ok = false;
                if (g) pend1 = true; else pend0 = true;
            }
        }
        if (!st->done) {
            const float alpha = (float)st->alpha;
            const int bx = wk.y % s.gx, jb = wk.y / s.gx;
            Acc<float> acc[2];
            if (s.colmode) {
                serve_prec_column(s, bx, jb, lane, w, alpha, acc);
            } else {
                // warp w: row w / nch of the item, chunk w % nch; warps past
                // rows * nch (and an item whose copies did not land) only take
                // part in the barriers
                const int row = w / s.nch, ch = w - row * s.nch;
                const int j = (landed && row < s.rows) ? jb * s.rows + row : s.op.ny;
                const Col<float> col = make_col(s.op, bx * 32 + lane, j);
                if (was_staged && s.ptab) {
                    // one factor set: the chunk-carry weights from the request's tables
                    const int nz = s.op.nz;
                    for (int k = tid; k < nz; k += 256) {
                        tb.g[k] = s.ptab[k];
                        tb.E[k] = s.ptab[nz + k];
                        tb.e[k] = s.ptab[2 * nz + k];
                        tb.C[k] = s.ptab[3 * nz + k];
                        tb.Q[k] = s.ptab[4 * nz + k];
                    }
                    __syncthreads();
                    const float* rs = sbase + g * 2 * SERVE_PVN + ((ch * SERVE_LZ) * s.rows + row) * 32 + lane;
                    if (s.rows == 1)
                        serve_prec_tab<1>(s, tb, col, lane, ch, row, alpha, acc, sh_y, sh_c, sh_z, sh_d, rs);
                    else if (s.rows == 2)
                        serve_prec_tab<2>(s, tb, col, lane, ch, row, alpha, acc, sh_y, sh_c, sh_z, sh_d, rs);
                    else
                        serve_prec_tab<4>(s, tb, col, lane, ch, row, alpha, acc, sh_y, sh_c, sh_z, sh_d, rs);
                } else {
                    const float* rs = was_staged
                        ? sbase + g * 2 * SERVE_PVN + ((ch * SERVE_LZ) * s.rows + row) * 32 + lane : nullptr;
                    serve_prec_generic(s, col, lane, ch, row, alpha, acc, sh_y, sh_c, sh_z, sh_d, rs);
                }
            }
            block_partials<2>(acc, s.partials + 2LL * wk.y);
        }
        __syncthreads();   // the stage has been read: refill it with the next item drawn
        if (tid == 0) issue(g);
    }
    // copies that did not land in time are waited for (again with a limit)
    // before the block's shared memory is released; an issued copy whose item
    // this block never reached cannot exist (a block's draws increase, and the
    // loop ends at the first draw past the end of the list)
    if (pend0) mbar_wait(bar0, par0, 1 << 22);
    if (pend1) mbar_wait(bar1, par1, 1 << 22);
}

// The SpMV items are taken in arrival order from `fetch` (zeroed before the
// launch), so blocks that draw cheap items (requests that stopped earlier in
// the graph, short columns) take more of them.  Two stages: thread 0 draws the
// item after next and starts its bulk copies as soon as a stage has been
// read, so one item's copies are in flight while the other is computed.  The
// tile arithmetic is that of k_sweep_spmv_tma2 (wrapped neighbours patched
// into the halo, level tables in shared memory, sigma per 16-level chunk).
constexpr size_t SERVE_SPMV_SMEM =
    2 * ((size_t)SpmvTmaTile<SERVE_LZ, SERVE_BY>::ZN + 3 * SpmvTmaTile<SERVE_LZ, SERVE_BY>::VN) * 4 + 16 + 128;

__global__ __launch_bounds__(BX * SERVE_BY) void k_serve_spmv(const ServeSlot* __restrict__ slots,
                                                             const int2* __restrict__ items,
                                                             const int* __restrict__ n_items,
                                                             unsigned* __restrict__ fetch) {
    using TT = SpmvTmaTile<SERVE_LZ, SERVE_BY>;
    constexpr int STAGE = TT::ZN + 3 * TT::VN;
    __shared__ int s_item[2];       // the item drawn for stage g (n or more: none)
    __shared__ int staged[2];       // stage g holds the bulk copies of its item (1) or nothing (0)
    __shared__ float tb[3][SERVE_LZ + 1];
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* sbase = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint64_t* bars = reinterpret_cast<uint64_t*>(sbase + 2 * STAGE);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    const uint32_t bar0 = smem_u32(bars), bar1 = smem_u32(bars + 1);
    const int n = *n_items;
    int last_slot = -1;   // thread 0: the slot whose maps it acquired last
    bool ok = true;       // false once a copy failed to land in time: no more copies are started
    // thread 0: draw the next item for stage g and start its copies if its
    // request has maps and is running
    auto issue = [&](int g) {
        const int it = (int)atomicAdd(fetch, 1u);
        s_item[g] = it;
        int go = 0;
        if (ok && it < n) {
            const int2 wk = items[it];
            const ServeSlot& sl = slots[wk.x];
            if (sl.tmaps && !sl.st->done) {
                if (wk.x != last_slot) {
                    for (int m = 0; m < 4; ++m) tmap_acquire(sl.tmaps + m);
                    last_slot = wk.x;
                }
                const int ch = wk.y % sl.nch, tile = wk.y / sl.nch;
                const int i0 = (tile % sl.gx) * BX, j0 = (tile / sl.gx) * SERVE_BY, k0 = ch * SERVE_LZ;
                float* zs = sbase + g * STAGE;
                const uint32_t bar = g ? bar1 : bar0;
                // earlier items used the stage through the generic proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect(bar, TT::BYTES);
                tma_load_3d(smem_u32(zs), sl.tmaps + 3, i0 - TMA_HALO_X, j0 - 1, k0 - 1, bar);
                tma_load_3d(smem_u32(zs + TT::ZN), sl.tmaps + 0, i0, j0, k0, bar);
                tma_load_3d(smem_u32(zs + TT::ZN + TT::VN), sl.tmaps + 1, i0, j0, k0, bar);
                tma_load_3d(smem_u32(zs + TT::ZN + 2 * TT::VN), sl.tmaps + 2, i0, j0, k0, bar);
                go = 1;
            }
        }
        staged[g] = go;
    };
    if (tid == 0) {
        mbar_init(bar0);
        mbar_init(bar1);
        issue(0);
        issue(1);
    }
    __syncthreads();
    uint32_t par0 = 0, par1 = 0;
    bool pend0 = false, pend1 = false;   // a copy into the stage that has not been seen to land
    for (int k = 0;; ++k) {
        const int g = k & 1;
        // s_item[g] and staged[g] were written before the barrier that ended the previous item
        const int it = s_item[g];
        if (it >= n) break;
        const int2 wk = items[it];
        const ServeSlot& sl = slots[wk.x];
        SolveState* st = sl.st;
        const bool was_staged = staged[g] != 0;
        const bool run = !st->done;        // the same for every thread: only this request's last item changes it
        const OpView<float>& op = sl.op;
        const int ch = wk.y % sl.nch, tile = wk.y / sl.nch;
        const int i0 = (tile % sl.gx) * BX, j0 = (tile / sl.gx) * SERVE_BY, k0 = ch * SERVE_LZ;
        const int kn = min(SERVE_LZ, op.nz - k0);
        float* zs = sbase + g * STAGE;
        float* us = zs + TT::ZN;
        float* ps = us + TT::VN;
        float* qs = ps + TT::VN;
        Col<float> col;
        WrapPatch<SERVE_LZ, SERVE_BY> wp;
        if (run) {
            // level tables, column geometry and wrapped neighbours while the copies fly
            if (tid < 3 * (SERVE_LZ + 1)) {
                const int a = tid / (SERVE_LZ + 1), t = tid - a * (SERVE_LZ + 1);
                const int kk = a == 0 ? k0 - 1 + t : k0 + t;
                const float* src = a == 0 ? op.wv : (a == 1 ? op.dk : op.mass);
                tb[a][t] = (kk >= 0 && kk < op.nz) ? ldro(src + kk) : 0.f;
            }
            col = make_col(op, i0 + tx, j0 + ty);
            wp.load(op, sl.z, i0, j0, k0, kn, tx, ty);
        }
        bool landed = ok;
        if (was_staged) {
            // a staged copy is always waited for before its stage can be refilled
            const bool l = mbar_wait(g ? bar1 : bar0, g ? par1 : par0, 1 << 22);
            landed = __syncthreads_and(l ? 1 : 0) != 0;
            if (landed) {
                if (g) par1 ^= 1u; else par0 ^= 1u;
            } else {
                if (g) pend1 = true; else pend0 = true;
            }
        }
        if (run) {
            if (!was_staged && ok) {
                // staged by the threads, cells outside the grid as zeros
                constexpr int NTH = BX * SERVE_BY;
                for (int e = tid; e < TT::ZN; e += NTH) {
                    const int xx = e % TT::ZX, yy = (e / TT::ZX) % TT::ZY, zz = e / (TT::ZX * TT::ZY);
                    const int gi = i0 - TMA_HALO_X + xx, gj = j0 - 1 + yy, gk = k0 - 1 + zz;
                    const bool in = gi >= 0 && gi < op.nx && gj >= 0 && gj < op.ny && gk >= 0 && gk < op.nz;
                    zs[e] = in ? ldro(sl.z + (long long)gk * op.plane + (long long)gj * op.nx + gi) : 0.f;
                }
                for (int e = tid; e < TT::VN; e += NTH) {
                    const int xx = e % BX, yy = (e / BX) % SERVE_BY, zz = e / (BX * SERVE_BY);
                    const int gi = i0 + xx, gj = j0 + yy, gk = k0 + zz;
                    const bool in = gi < op.nx && gj < op.ny && gk < op.nz;
                    const long long o = (long long)gk * op.plane + (long long)gj * op.nx + gi;
                    us[e] = in ? sl.u[o] : 0.f;
                    ps[e] = in ? sl.p[o] : 0.f;
                    qs[e] = in ? sl.q[o] : 0.f;
                }
            }
            if (!landed) {
                if (tid == 0) atomicExch(&st->status, 6);   // PCG_TIMEOUT: this item is not computed
                ok = false;
            } else {
                wp.store(zs, tx, ty);
            }
            __syncthreads();
            Acc<float> sig[1];
            if (landed && col.valid && kn > 0)
                spmv_tile_compute_p<SERVE_LZ, SERVE_BY>(op, col, tx, ty, k0, kn, zs, us, ps, qs, &tb[0][1], tb[1],
                                                        tb[2], sl.u, sl.p, sl.q, (float)st->alpha, (float)st->beta,
                                                        sig[0]);
            block_partials<1>(sig, sl.partials + wk.y);
        } else if (was_staged && !landed) {
            ok = false;
        }
        __syncthreads();   // the stage and the tables have been read: refill with the next item drawn
        if (tid == 0) issue(g);
    }
    // copies that did not land in time are waited for (again with a limit)
    // before the block's shared memory is released
    if (pend0) mbar_wait(bar0, par0, 1 << 22);
    if (pend1) mbar_wait(bar1, par1, 1 << 22);
}

// The scalar steps of an epoch's sweep for every request in its inner phase,
// one block per slot (PH 0: after the preconditioner sweep, PH 1: after the
// SpMV sweep): the items' partial sums added in a fixed order (so a request's
// scalars do not depend on the other requests of the batch), then the
// epilogue of the one-request sweeps.  A request that had stopped before the
// launch wrote no partials and is skipped.
template <int PH>
__global__ __launch_bounds__(256) void k_serve_scalars(const ServeSlot* __restrict__ slots,
                                                       const int* __restrict__ inner) {
    constexpr int N = PH == 0 ? 2 : 1;
    __shared__ double tot[N][MAXW];
    const int slot = blockIdx.x;
    if (!inner[slot]) return;
    const ServeSlot& s = slots[slot];
    SolveState* st = s.st;
    if (st->done) return;
    const int nb = PH == 0 ? s.nprec : s.nspmv;
    double acc[N];
#pragma unroll
    for (int n = 0; n < N; ++n) acc[n] = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
#pragma unroll
        for (int n = 0; n < N; ++n) acc[n] += __ldcg(s.partials + (long long)b * N + n);
    }
    block_sum<N>(acc, tot);
    if (threadIdx.x == 0) {
        if (PH == 0) prec_epilogue(st, acc[0], acc[N - 1]);
        else spmv_epilogue(st, acc[0]);
    }
}

}  // namespace pcg
