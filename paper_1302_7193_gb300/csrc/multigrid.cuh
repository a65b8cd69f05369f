// Device kernels of the multigrid preconditioner (PCG_PREC_MULTIGRID).
//
// A V-cycle on a hierarchy of horizontally coarsened grids (the solver the
// paper names as the next step, Section 8): damped block-Jacobi smoothing
// with the column blocks of each level (Thomas recurrences in the excess
// form of kernels.cuh), residuals in flux form, restriction by summing the
// four fine cells of a coarse cell and prolongation by its transpose.  The
// V-cycle kernels are templated on the precision T of the cycle (FP64, or
// FP32 inside the FP64 CG of PCG_PREC_MULTIGRID_F32); the CG steps around
// it are FP64.
#pragma once
#include "kernels.cuh"

namespace pcg {

// ---------------------------------------------------------------------------
// Multigrid V-cycle on a hierarchy of horizontally coarsened grids:
// damped block-Jacobi smoothing with the column blocks, residuals, and the
// transfers R (sum of the four fine cells of a coarse cell) and P = R^T.
// Every kernel skips a right-hand side whose solve has stopped (st[rhs].done).
// ---------------------------------------------------------------------------
// z = (acc ? z : 0) + omega M^{-1} rin, one thread per column; tmp receives
// the forward sweep's y_k (tmp may be rin itself).  The Thomas recurrences
// run in the excess form (g_k = 1/D_k, E_k = D_k - W_k):
//   y_k = (r_k - e_{k-1} y_{k-1}) + y_{k-1},  e = E g,
//   z_k = z_{k+1} + g_k (y_k - E_k z_{k+1}),
// because on coarse levels the vertical couplings grow 4x per level against
// the horizontal ones, the excess 1 - W/D falls towards 1e-7 and a stored
// ratio W/D would carry it with a relative error of 2^-53 / (1 - W/D).
template <typename T>
__global__ __launch_bounds__(NT) void k_mg_smooth(OpView<T> op, const T* rin, T* tmp, T* z, T omega, int acc,
                                                  const SolveState* __restrict__ st) {
    const int rhs = blockIdx.z;
    if (st[rhs].done) return;
    const Col<T> col = make_col(op, blockIdx.x * BX + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
    if (!col.valid) return;
    const long long base = (long long)rhs * op.vol + col.c;
    const long long pl = op.plane, fs = op.ncls;
    const T* fg = op.fg + col.cls;
    const T* fe = op.fe + col.cls;
    const int nz = op.nz;
    // the loads of the next PB levels are issued before the current PB levels
    // are stored (tmp may be rin, and z is read and written)
    constexpr int PB = 8;
    T y = T(0), eprev = T(0);
    T ra[PB];
#pragma unroll
    for (int t = 0; t < PB; ++t) ra[t] = t < nz ? rin[base + t * pl] : T(0);
    for (int k0 = 0; k0 < nz; k0 += PB) {
        T rn[PB];
#pragma unroll
        for (int t = 0; t < PB; ++t) {
            const int k = k0 + PB + t;
            rn[t] = k < nz ? rin[base + k * pl] : T(0);
        }
#pragma unroll
        for (int t = 0; t < PB; ++t) {
            const int k = k0 + t;
            if (k < nz) {
                y = fma(-eprev, y, ra[t]) + y;
                tmp[base + k * pl] = y;
                eprev = ldro(fe + k * fs) * ldro(fg + k * fs);
            }
        }
#pragma unroll
        for (int t = 0; t < PB; ++t) ra[t] = rn[t];
    }
    T zn = T(0);
    T ya[PB], za[PB];
    const int kt = nz - 1;
#pragma unroll
    for (int t = 0; t < PB; ++t) {
        const int k = kt - t;
        ya[t] = k >= 0 ? tmp[base + k * pl] : T(0);
        za[t] = (acc && k >= 0) ? z[base + k * pl] : T(0);
    }
    for (int k0 = kt; k0 >= 0; k0 -= PB) {
        T yn[PB], zn_[PB];
#pragma unroll
        for (int t = 0; t < PB; ++t) {
            const int k = k0 - PB - t;
            yn[t] = k >= 0 ? tmp[base + k * pl] : T(0);
            zn_[t] = (acc && k >= 0) ? z[base + k * pl] : T(0);
        }
#pragma unroll
        for (int t = 0; t < PB; ++t) {
            const int k = k0 - t;
            if (k >= 0) {
                zn = fma(ldro(fg + k * fs), fma(-ldro(fe + k * fs), zn, ya[t]), zn);
                z[base + k * pl] = acc ? fma(omega, zn, za[t]) : omega * zn;
            }
        }
#pragma unroll
        for (int t = 0; t < PB; ++t) {
            ya[t] = yn[t];
            za[t] = zn_[t];
        }
    }
}

// t = r - A z (flux form, as k_apply).  blockIdx.z = rhs * ksplit + part:
// part takes levels [part n_z / ksplit, (part + 1) n_z / ksplit) of every
// column (a column's levels are independent here apart from the flux carried
// from below, which the part recomputes), so that enough threads run to keep
// the loads in flight.  Each thread issues the loads of its next PB levels
// (the column, its four neighbours, r) before it computes the current PB.
template <typename T, int PB>
__global__ __launch_bounds__(NT) void k_mg_resid(OpView<T> op, const T* __restrict__ r, const T* __restrict__ z,
                                                 T* __restrict__ t, const SolveState* __restrict__ st, int ksplit) {
    const int rhs = blockIdx.z / ksplit;
    const int part = blockIdx.z - rhs * ksplit;
    if (st[rhs].done) return;
    const Col<T> col = make_col(op, blockIdx.x * BX + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
    if (!col.valid) return;
    const int nz = op.nz;
    const int k0 = (int)((long long)part * nz / ksplit), k1 = (int)((long long)(part + 1) * nz / ksplit);
    const long long pl = op.plane, base = (long long)rhs * op.vol;
    const T* __restrict__ zb = z + base;
    const T* __restrict__ rb = r + base + col.c;
    T* __restrict__ tb = t + base + col.c;
    T qz[PB], qe[PB], qw[PB], qn[PB], qs[PB], qr[PB];
    auto fetch = [&](int kb, T(&vz)[PB], T(&ve)[PB], T(&vw)[PB], T(&vn)[PB], T(&vs)[PB], T(&vr)[PB]) {
#pragma unroll
        for (int u = 0; u < PB; ++u) {
            const int k = kb + u;
            if (k < k1) {
                const T* zl = zb + (long long)k * pl;
                vz[u] = ldro(zl + col.c);
                ve[u] = ldro(zl + col.ce);
                vw[u] = ldro(zl + col.cw);
                vn[u] = ldro(zl + col.cn);
                vs[u] = ldro(zl + col.cs);
                vr[u] = rb[(long long)k * pl];
            }
        }
    };
    fetch(k0, qz, qe, qw, qn, qs, qr);
    const T zend = k1 < nz ? ldro(zb + (long long)k1 * pl + col.c) : T(0);   // the level above the part
    T fprev = k0 > 0 ? ldro(op.wv + k0 - 1) * (ldro(zb + (long long)(k0 - 1) * pl + col.c) - qz[0]) : T(0);
    for (int kb = k0; kb < k1; kb += PB) {
        T xz[PB], xe[PB], xw[PB], xn[PB], xs[PB], xr[PB];
        fetch(kb + PB, xz, xe, xw, xn, xs, xr);
#pragma unroll
        for (int u = 0; u < PB; ++u) {
            const int k = kb + u;
            if (k < k1) {
                const T zc = qz[u];
                const T zu = (k + 1 < k1) ? (u + 1 < PB ? qz[u + 1] : xz[0]) : (k1 < nz ? zend : zc);
                const T f = ldro(op.wv + k) * (zc - zu);
                T h = col.me * (zc - qe[u]);
                h = fma(col.mw, zc - qw[u], h);
                h = fma(col.mn, zc - qn[u], h);
                h = fma(col.ms, zc - qs[u], h);
                const T az = fma(ldro(op.dk + k), h, col.area * fma(ldro(op.mass + k), zc, f - fprev));
                tb[(long long)k * pl] = qr[u] - az;
                fprev = f;
            }
        }
#pragma unroll
        for (int u = 0; u < PB; ++u) {
            qz[u] = xz[u];
            qe[u] = xe[u];
            qw[u] = xw[u];
            qn[u] = xn[u];
            qs[u] = xs[u];
            qr[u] = xr[u];
        }
    }
}

// rc = R (r - A z): the residual of the downward leg, restricted as it is
// formed (k_mg_resid followed by k_mg_restrict, without writing t).  Blocks of
// 32 x 2 fine columns (an even pair of rows; n_x and n_y are even on every
// level that is restricted); blockIdx.z = rhs * ksplit + part as in
// k_mg_resid.  Each coarse cell sums its four fine residuals in the order of
// k_mg_restrict, ((t(2J,2I) + t(2J,2I+1)) + t(2J+1,2I)) + t(2J+1,2I+1): the
// x pair by a shuffle, the row 2J+1 values through shared memory once per PB
// levels.
template <typename T, int PB>
__global__ __launch_bounds__(64) void k_mg_resid_restrict(OpView<T> op, const T* __restrict__ r,
                                                          const T* __restrict__ z, T* __restrict__ rc,
                                                          const SolveState* __restrict__ st, int ksplit) {
    __shared__ T sh[PB][32];
    const int rhs = blockIdx.z / ksplit;
    const int part = blockIdx.z - rhs * ksplit;
    if (st[rhs].done) return;
    const int lane = threadIdx.x, ty = threadIdx.y;
    const Col<T> col = make_col(op, blockIdx.x * 32 + lane, blockIdx.y * 2 + ty);
    const int nz = op.nz;
    const int k0 = (int)((long long)part * nz / ksplit), k1 = (int)((long long)(part + 1) * nz / ksplit);
    const long long pl = op.plane, base = (long long)rhs * op.vol;
    const T* __restrict__ zb = z + base;
    const T* __restrict__ rb = r + base + col.c;
    const int nxc = op.nx / 2;
    const long long planec = pl / 4;
    const int ic = blockIdx.x * 16 + lane / 2, jc = blockIdx.y;
    T* __restrict__ rcb = rc + (long long)rhs * planec * nz + (long long)jc * nxc + ic;
    T qz[PB], qe[PB], qw[PB], qn[PB], qs[PB], qr[PB];
    // lanes outside the grid (levels narrower than 32 columns) load nothing
    // and contribute zeros, but take part in the shuffles and barriers
    auto fetch = [&](int kb, T(&vz)[PB], T(&ve)[PB], T(&vw)[PB], T(&vn)[PB], T(&vs)[PB], T(&vr)[PB]) {
#pragma unroll
        for (int u = 0; u < PB; ++u) {
            const int k = kb + u;
            if (col.valid && k < k1) {
                const T* zl = zb + (long long)k * pl;
                vz[u] = ldro(zl + col.c);
                ve[u] = ldro(zl + col.ce);
                vw[u] = ldro(zl + col.cw);
                vn[u] = ldro(zl + col.cn);
                vs[u] = ldro(zl + col.cs);
                vr[u] = rb[(long long)k * pl];
            }
        }
    };
    fetch(k0, qz, qe, qw, qn, qs, qr);
    const T zend = (col.valid && k1 < nz) ? ldro(zb + (long long)k1 * pl + col.c) : T(0);
    T fprev = (col.valid && k0 > 0) ? ldro(op.wv + k0 - 1) * (ldro(zb + (long long)(k0 - 1) * pl + col.c) - qz[0]) : T(0);
    for (int kb = k0; kb < k1; kb += PB) {
        T xz[PB], xe[PB], xw[PB], xn[PB], xs[PB], xr[PB];
        fetch(kb + PB, xz, xe, xw, xn, xs, xr);
        T tv[PB];
#pragma unroll
        for (int u = 0; u < PB; ++u) {
            const int k = kb + u;
            tv[u] = T(0);
            if (col.valid && k < k1) {
                const T zc = qz[u];
                const T zu = (k + 1 < k1) ? (u + 1 < PB ? qz[u + 1] : xz[0]) : (k1 < nz ? zend : zc);
                const T f = ldro(op.wv + k) * (zc - zu);
                T h = col.me * (zc - qe[u]);
                h = fma(col.mw, zc - qw[u], h);
                h = fma(col.mn, zc - qn[u], h);
                h = fma(col.ms, zc - qs[u], h);
                const T az = fma(ldro(op.dk + k), h, col.area * fma(ldro(op.mass + k), zc, f - fprev));
                tv[u] = qr[u] - az;
                fprev = f;
            }
        }
        if (ty == 1) {
#pragma unroll
            for (int u = 0; u < PB; ++u) sh[u][lane] = tv[u];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PB; ++u) {
            const T right = __shfl_down_sync(0xffffffffu, tv[u], 1);
            const int k = kb + u;
            if (ty == 0 && !(lane & 1) && col.valid && k < k1)
                rcb[(long long)k * planec] = ((tv[u] + right) + sh[u][lane]) + sh[u][lane + 1];
        }
        __syncthreads();   // the rows 2J+1 of the next PB levels overwrite sh
#pragma unroll
        for (int u = 0; u < PB; ++u) {
            qz[u] = xz[u];
            qe[u] = xe[u];
            qw[u] = xw[u];
            qn[u] = xn[u];
            qs[u] = xs[u];
            qr[u] = xr[u];
        }
    }
}

// z = (acc ? z : 0) + omega M^{-1} rin on levels with few columns: the
// chunked (substructured) Thomas solve of prec_chunked_body, one warp per
// 16-level chunk of 32 columns of one row (block (32, n_z/16)), so that a
// column's work spreads over several warps; the damped update is its store.
template <typename T>
__global__ __launch_bounds__(256) void k_mg_lsolve_chunked(OpView<T> op, const T* rin, T* z, T omega, int acc,
                                                           const SolveState* __restrict__ st) {
    __shared__ T sh_y[MAXW][32], sh_c[MAXW][32], sh_z[MAXW][32], sh_d[MAXW][32];
    const int rhs = blockIdx.z;
    if (st[rhs].done) return;
    const int lane = threadIdx.x, ch = threadIdx.y, nch = blockDim.y;
    const Col<T> col = make_col(op, blockIdx.x * 32 + lane, blockIdx.y);
    const long long rb = (long long)rhs * op.vol;
    Acc<T> sums[2];
    // alpha = 0: the chunk's "updated residual" is rin itself, and it is not stored back
    if (acc)
        prec_chunked_body<T, 16, false, 2>(op, col, lane, ch, nch, 0, const_cast<T*>(rin + rb), rin + rb, z + rb, T(0),
                                           sums, sh_y, sh_c, sh_z, sh_d, nullptr, nullptr, 0, omega);
    else
        prec_chunked_body<T, 16, false, 1>(op, col, lane, ch, nch, 0, const_cast<T*>(rin + rb), rin + rb, z + rb, T(0),
                                           sums, sh_y, sh_c, sh_z, sh_d, nullptr, nullptr, 0, omega);
}

// Elementwise kernels run on a 2-D grid (x: cells of one right-hand side,
// grid-stride; y: right-hand sides), and the transfers on a 3-D grid (x: tiles
// of blockDim.x x blockDim.y cells of a level, y: levels, z: right-hand
// sides), so that no thread divides a flat cell index.  Right-hand sides
// whose solve has stopped are skipped.
template <class F>
__device__ __forceinline__ void for_each_elem(long long vol, int nrhs, const SolveState* __restrict__ st, F f) {
    for (int rhs = blockIdx.y; rhs < nrhs; rhs += gridDim.y) {
        if (st[rhs].done) continue;
        const long long b = (long long)rhs * vol;
        for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < vol; c += (long long)gridDim.x * blockDim.x)
            f(b + c, rhs);
    }
}

// f(rhs, k, j, i) for every cell of an (nrhs, nz, ny, nx) array; nbi = tiles per row of tiles
// (a thread takes every gridDim.y-th level: several independent loads in flight)
template <class F>
__device__ __forceinline__ void for_each_cell(int nx, int ny, int nz, int nrhs, int nbi,
                                              const SolveState* __restrict__ st, F f) {
    const int jb = blockIdx.x / nbi, ib = blockIdx.x - jb * nbi;
    const int i = ib * blockDim.x + threadIdx.x, j = jb * blockDim.y + threadIdx.y;
    if (i >= nx || j >= ny) return;
    for (int rhs = blockIdx.z; rhs < nrhs; rhs += gridDim.z) {
        if (st[rhs].done) continue;
#pragma unroll 4
        for (int k = blockIdx.y; k < nz; k += gridDim.y) f(rhs, k, j, i);
    }
}

// rc = R tf: every coarse cell (rhs, k, J, I) sums the fine cells
// (2J, 2I), (2J, 2I+1), (2J+1, 2I), (2J+1, 2I+1) of the same level k.
template <typename T>
__global__ void k_mg_restrict(const T* __restrict__ tf, T* __restrict__ rc, int nxc, int nyc, int nz, int nrhs,
                              int nbi, const SolveState* __restrict__ st) {
    const long long planec = (long long)nxc * nyc, volc = planec * nz;
    const long long nxf = 2LL * nxc, planef = 4 * planec;
    for_each_cell(nxc, nyc, nz, nrhs, nbi, st, [&](int rhs, int k, int jc, int ic) {
        const T* f = tf + rhs * (volc * 4) + k * planef + (2LL * jc) * nxf + 2 * ic;
        rc[rhs * volc + k * planec + (long long)jc * nxc + ic] = ((f[0] + f[1]) + f[nxf]) + f[nxf + 1];
    });
}

// zf += P zc: every fine cell adds its coarse cell's value.
template <typename T>
__global__ void k_mg_prolong(const T* __restrict__ zc, T* __restrict__ zf, int nxf, int nyf, int nz, int nrhs,
                             int nbi, const SolveState* __restrict__ st) {
    const long long planef = (long long)nxf * nyf, volf = planef * nz;
    const int nxc = nxf / 2;
    const long long planec = planef / 4, volc = planec * nz;
    for_each_cell(nxf, nyf, nz, nrhs, nbi, st, [&](int rhs, int k, int j, int i) {
        zf[rhs * volf + k * planef + (long long)j * nxf + i] +=
            zc[rhs * volc + k * planec + (long long)(j >> 1) * nxc + (i >> 1)];
    });
}

// a <-> b between the FP64 CG and an FP32 V-cycle
template <typename TA, typename TB>
__global__ void k_mg_convert(const TA* __restrict__ a, TB* __restrict__ b, long long vol, int nrhs,
                             const SolveState* __restrict__ st) {
    for_each_elem(vol, nrhs, st, [&](long long c, int) { b[c] = (TB)a[c]; });
}

// r <- r - alpha q (Algorithm 1 line 2, the preconditioner itself applied separately)
__global__ void k_mg_rupdate(double* __restrict__ r, const double* __restrict__ q, long long vol, int nrhs,
                             const SolveState* __restrict__ st) {
    for_each_elem(vol, nrhs, st, [&](long long c, int rhs) { r[c] = fma(-st[rhs].alpha, q[c], r[c]); });
}

// <r, r> and <r, z> of every right-hand side; the last block applies the
// stopping test and forms beta (Algorithm 1 lines 3-4, as k_sweep_prec).
__global__ __launch_bounds__(NT) void k_mg_dots(OpView<double> op, const double* __restrict__ r,
                                                const double* __restrict__ z, SolveState* __restrict__ states,
                                                double* __restrict__ partials, unsigned* __restrict__ counters,
                                                int nblocks) {
    const int rhs = blockIdx.z;
    SolveState* st = states + rhs;
    if (st->done) return;
    const Col<double> col = make_col(op, blockIdx.x * BX + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
    Acc<double> acc[2];
    if (col.valid) {
        const long long base = (long long)rhs * op.vol + col.c;
        for (int k = 0; k < op.nz; ++k) {
            const long long o = base + (long long)k * op.plane;
            const double rk = r[o];
            acc[0].add_prod(rk, rk);
            acc[1].add_prod(rk, z[o]);
        }
    }
    double v[2];
    if (grid_sum_acc<2>(acc, partials + (long long)rhs * nblocks * 2, counters + rhs, nblocks, bid2(), v))
        prec_epilogue(st, v[0], v[1]);
}

}  // namespace pcg
