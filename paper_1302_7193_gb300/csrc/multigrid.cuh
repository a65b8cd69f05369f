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

// zf += P zc on FP32 levels whose rows split into quads (n_x % 4 == 0, n_y
// even): a thread adds the two coarse values under a quad of fine cells, at
// every gridDim.y-th level.  Grid (ceil(n_y n_x / 4 / 256), level groups, nrhs).
__global__ __launch_bounds__(256) void k_mg_prolong4(const float* __restrict__ zc, float* __restrict__ zf, int nxf,
                                                     int nyf, int nz, int nrhs, const SolveState* __restrict__ st) {
    const int nq = nxf / 4;
    const long long u = (long long)blockIdx.x * 256 + threadIdx.x;
    if (u >= (long long)nyf * nq) return;
    const int j = (int)(u / nq), q = (int)(u - (long long)j * nq);
    const long long planef = (long long)nxf * nyf, planec = planef / 4;
    const int nxc = nxf / 2;
    for (int rhs = blockIdx.z; rhs < nrhs; rhs += gridDim.z) {
        if (st[rhs].done) continue;
        float* f = zf + rhs * planef * nz + (long long)j * nxf + 4 * q;
        const float* c = zc + rhs * planec * nz + (long long)(j >> 1) * nxc + 2 * q;
#pragma unroll 4
        for (int k = blockIdx.y; k < nz; k += gridDim.y) {
            float4 v = *reinterpret_cast<float4*>(f + k * planef);
            const float2 p = __ldg(reinterpret_cast<const float2*>(c + k * planec));
            v.x += p.x;
            v.y += p.x;
            v.z += p.y;
            v.w += p.y;
            *reinterpret_cast<float4*>(f + k * planef) = v;
        }
    }
}

// a <-> b between the FP64 CG and an FP32 V-cycle
template <typename TA, typename TB>
__global__ void k_mg_convert(const TA* __restrict__ a, TB* __restrict__ b, long long vol, int nrhs,
                             const SolveState* __restrict__ st) {
    for_each_elem(vol, nrhs, st, [&](long long c, int) { b[c] = (TB)a[c]; });
}

// r <- r - alpha q (Algorithm 1 line 2, the preconditioner itself applied
// separately); rf, if not null, receives r rounded to FP32 (the input of an
// FP32 V-cycle).
__global__ void k_mg_rupdate(double* __restrict__ r, const double* __restrict__ q, float* __restrict__ rf,
                             long long vol, int nrhs, const SolveState* __restrict__ st) {
    for_each_elem(vol, nrhs, st, [&](long long c, int rhs) {
        const double v = fma(-st[rhs].alpha, q[c], r[c]);
        r[c] = v;
        if (rf) rf[c] = (float)v;
    });
}

// <r, r> and <r, z> of every right-hand side; the last block applies the
// stopping test and forms beta (Algorithm 1 lines 3-4, as k_sweep_prec).
// With zf (an FP32 V-cycle's output) z is first widened from it and stored.
__global__ __launch_bounds__(NT) void k_mg_dots(OpView<double> op, const double* __restrict__ r,
                                                double* __restrict__ z, const float* __restrict__ zf,
                                                SolveState* __restrict__ states, double* __restrict__ partials,
                                                unsigned* __restrict__ counters, int nblocks) {
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
            double zk;
            if (zf) {
                zk = (double)zf[o];
                z[o] = zk;
            } else {
                zk = z[o];
            }
            acc[0].add_prod(rk, rk);
            acc[1].add_prod(rk, zk);
        }
    }
    double v[2];
    if (grid_sum_acc<2>(acc, partials + (long long)rhs * nblocks * 2, counters + rhs, nblocks, bid2(), v))
        prec_epilogue(st, v[0], v[1]);
}

// ---------------------------------------------------------------------------
// FP32 residuals on levels whose rows split into quads (n_x % 4 == 0; n_y is
// even on every level but the coarsest).  A thread takes the four cells
// i0 .. i0+3 of both rows of a row pair (2 jp, 2 jp + 1): the pair's own z
// rows are each other's north and south neighbours, the east and west
// neighbours at a quad's edges come from the adjacent lanes by shuffles
// (loads only at the ends of rows and warps), and z, r move as float4.  Each
// cell's arithmetic is that of k_mg_resid, in the same order.
//   MODE 0: t = r - A z
//   MODE 1: rc = R (r - A z), the four fine residuals of a coarse cell summed
//           in the order of k_mg_restrict (t is not stored)
// Grid (ceil(units / 128), 1, nrhs * ksplit), units = (n_y / 2) (n_x / 4);
// blockIdx.z = rhs * ksplit + part, part taking levels
// [part n_z / ksplit, (part + 1) n_z / ksplit).
// ---------------------------------------------------------------------------
// A row pair's two quads at one level: the own z rows, needed one level
// earlier too (as the level above), and the rest.
struct QuadOwn {
    float4 z0, z1;     // rows 2 jp, 2 jp + 1
};
struct QuadRest {
    float4 zs, zn;     // the row below 2 jp, the row above 2 jp + 1
    float4 r0, r1;
    float e0, w0, e1, w1;   // edge neighbours where no lane holds them
};

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float q4(const float4& v, int m) {
    return m == 0 ? v.x : (m == 1 ? v.y : (m == 2 ? v.z : v.w));
}

template <int MODE>
__global__ __launch_bounds__(128) void k_mg_resid4(OpView<float> op, const float* __restrict__ r,
                                                   const float* __restrict__ z, float* __restrict__ out,
                                                   const SolveState* __restrict__ st, int ksplit) {
    const int rhs = blockIdx.z / ksplit;
    const int part = blockIdx.z - rhs * ksplit;
    if (st[rhs].done) return;   // the same for the whole block
    const int lane = threadIdx.x & 31;
    const int nx = op.nx, ny = op.ny, nz = op.nz, nq = nx / 4;
    const int units = (ny / 2) * nq;
    const int u = blockIdx.x * 128 + threadIdx.x;
    const bool valid = u < units;   // invalid threads still join the shuffles
    const int jp = valid ? u / nq : 0;
    const int q = valid ? u - jp * nq : 0;
    const int j0 = 2 * jp, j1 = j0 + 1, i0 = 4 * q;
    const int js = j0 > 0 ? j0 - 1 : (op.periodic_y ? ny - 1 : 0);
    const int jn = j1 + 1 < ny ? j1 + 1 : (op.periodic_y ? 0 : j1);
    const int ie = i0 + 4 < nx ? i0 + 4 : 0, iw = i0 > 0 ? i0 - 1 : nx - 1;
    const bool e_shfl = q + 1 < nq && lane < 31, w_shfl = q > 0 && lane > 0;
    const long long pl = op.plane, c0 = (long long)j0 * nx + i0, c1 = c0 + nx;
    const long long cs = (long long)js * nx + i0, cn = (long long)jn * nx + i0;
    const int nxc = nx / 2;
    const long long plc = pl / 4;
    const long long base = (long long)rhs * op.vol;
    const float* __restrict__ zb = z + base;
    const float* __restrict__ rb = r + base;
    const int k0 = (int)((long long)part * nz / ksplit), k1 = (int)((long long)(part + 1) * nz / ksplit);
    auto zq = [&](int k, long long c) -> float4 { return ld4(zb + (long long)k * pl + c); };   // a quad of z
    auto zpt = [&](int k, int j, int i) -> float { return __ldg(zb + (long long)k * pl + (long long)j * nx + i); };
    // a level's loads: the own rows are issued three levels ahead (the level
    // above is read one level before the level itself), the rest two
    auto fetch_own = [&](int k, QuadOwn& v) {
        if (!valid) return;
        v.z0 = zq(k, c0);
        v.z1 = zq(k, c1);
    };
    auto fetch_rest = [&](int k, QuadRest& v) {
        if (!valid) return;
        v.zs = zq(k, cs);
        v.zn = zq(k, cn);
        v.r0 = ld4(rb + (long long)k * pl + c0);
        v.r1 = ld4(rb + (long long)k * pl + c1);
        if (!e_shfl) {
            v.e0 = zpt(k, j0, ie);
            v.e1 = zpt(k, j1, ie);
        }
        if (!w_shfl) {
            v.w0 = zpt(k, j0, iw);
            v.w1 = zpt(k, j1, iw);
        }
    };
    // face weights of the eight cells, as make_col forms them (scalar loads:
    // the tables are not aligned for vector loads)
    float me[2][4], mw[2][4], mn[2][4], ms[2][4], ar[2][4];
    {
        const long long cr[2] = {c0, c1};
        const int jr[2] = {j0, j1};
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                me[h][m] = valid ? ldro(op.mue + cr[h] + m) : 0.f;
                mn[h][m] = valid ? ldro(op.mun + cr[h] + m) : 0.f;
                ar[h][m] = valid ? ldro(op.area + (op.area_percol ? cr[h] + m : (long long)jr[h])) : 0.f;
            }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float wsh = __shfl_up_sync(0xffffffffu, me[h][3], 1);
            mw[h][0] = w_shfl ? wsh : (valid ? ldro(op.mue + (long long)jr[h] * nx + iw) : 0.f);
#pragma unroll
            for (int m = 1; m < 4; ++m) mw[h][m] = me[h][m - 1];
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            ms[0][m] = (valid && (op.periodic_y || j0 > 0)) ? ldro(op.mun + cs + m) : 0.f;
            ms[1][m] = mn[0][m];
        }
    }
    // own rows of levels k .. k + 3 (up to k1, the level above the part,
    // below n_z), the rest of levels k .. k + 2 (below k1)
    QuadOwn o0{}, o1{}, o2{}, o3{};
    QuadRest q0{}, q1{}, q2{};
    const int kown = min(k1, nz - 1);
    fetch_own(k0, o0);
    if (k0 + 1 <= kown) fetch_own(k0 + 1, o1);
    if (k0 + 2 <= kown) fetch_own(k0 + 2, o2);
    fetch_rest(k0, q0);
    if (k0 + 1 < k1) fetch_rest(k0 + 1, q1);
    float fp[2][4];   // vertical flux from below, per cell
    if (k0 > 0) {
        QuadOwn lo{};
        fetch_own(k0 - 1, lo);
        const float wlo = ldro(op.wv + k0 - 1);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            fp[0][m] = wlo * (q4(lo.z0, m) - q4(o0.z0, m));
            fp[1][m] = wlo * (q4(lo.z1, m) - q4(o0.z1, m));
        }
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) fp[0][m] = fp[1][m] = 0.f;
    }
    for (int k = k0; k < k1; ++k) {
        if (k + 3 <= kown) fetch_own(k + 3, o3);
        if (k + 2 < k1) fetch_rest(k + 2, q2);
        const float wvk = ldro(op.wv + k), dkk = ldro(op.dk + k), mk = ldro(op.mass + k);
        const bool top = k + 1 >= nz;
        float t[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 zr = h == 0 ? o0.z0 : o0.z1;
            const float4 zup = h == 0 ? o1.z0 : o1.z1;
            const float4 zno = h == 0 ? o0.z1 : q0.zn;   // north row
            const float4 zso = h == 0 ? q0.zs : o0.z0;   // south row
            const float4 rr = h == 0 ? q0.r0 : q0.r1;
            const float esh = __shfl_down_sync(0xffffffffu, zr.x, 1);
            const float wsh = __shfl_up_sync(0xffffffffu, zr.w, 1);
            const float E = e_shfl ? esh : (h == 0 ? q0.e0 : q0.e1);
            const float Wv = w_shfl ? wsh : (h == 0 ? q0.w0 : q0.w1);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float zcv = q4(zr, m);
                const float zu = top ? zcv : q4(zup, m);
                const float ze = m < 3 ? q4(zr, m + 1) : E;
                const float zw = m > 0 ? q4(zr, m - 1) : Wv;
                const float f = wvk * (zcv - zu);
                float hh = me[h][m] * (zcv - ze);
                hh = fmaf(mw[h][m], zcv - zw, hh);
                hh = fmaf(mn[h][m], zcv - q4(zno, m), hh);
                hh = fmaf(ms[h][m], zcv - q4(zso, m), hh);
                const float az = fmaf(dkk, hh, ar[h][m] * fmaf(mk, zcv, f - fp[h][m]));
                t[h][m] = q4(rr, m) - az;
                fp[h][m] = f;
            }
        }
        if (valid) {
            if constexpr (MODE == 1) {
                float2 v;
                v.x = ((t[0][0] + t[0][1]) + t[1][0]) + t[1][1];
                v.y = ((t[0][2] + t[0][3]) + t[1][2]) + t[1][3];
                *reinterpret_cast<float2*>(out + (long long)rhs * (op.vol / 4) + (long long)k * plc +
                                           (long long)jp * nxc + 2 * q) = v;
            } else {
                float* ob = out + base + (long long)k * pl;
                *reinterpret_cast<float4*>(ob + c0) = make_float4(t[0][0], t[0][1], t[0][2], t[0][3]);
                *reinterpret_cast<float4*>(ob + c1) = make_float4(t[1][0], t[1][1], t[1][2], t[1][3]);
            }
        }
        o0 = o1;
        o1 = o2;
        o2 = o3;
        q0 = q1;
        q1 = q2;
    }
}

// ---------------------------------------------------------------------------
// The coarse end of the V-cycle in one launch.
//
// On the smallest levels every step of the cycle is a short chain of
// dependent work on a few thousand cells, and a launch per step costs
// several microseconds of fill, first loads and drain whatever the level's
// size.  k_mg_tail runs the levels lt .. L-1 -- the downward smoothing and
// restriction, the coarsest level, the prolongation and the upward smoothing
// back to lt -- in one thread block per right-hand side, with the levels'
// vectors held in shared memory (r and z of every level, one residual
// scratch of the largest) and a block barrier between dependent steps.  It
// reads r of level lt from global memory at the start and writes z of level
// lt back at the end.  Every step does the arithmetic of the kernel it
// replaces in the same order (the chunked line solve of k_mg_lsolve_chunked,
// the flux-form residual of k_mg_resid, the four-cell sums of k_mg_restrict
// and k_mg_prolong), so the cycle's result does not depend on where the
// tail starts.
// ---------------------------------------------------------------------------
constexpr int TAIL_MAXL = 8;
constexpr int TAIL_WARPS = 8;   // 256 threads: the chunked line solve's registers

template <typename T>
struct TailArgs {
    OpView<T> op[TAIL_MAXL];          // levels lt .. L-1
    long long off_r[TAIL_MAXL];       // r of each level in the dynamic shared memory (elements)
    long long off_z[TAIL_MAXL];       // z of each level
    long long off_t;                  // residual scratch (the largest level's size)
    const T* r_in;                    // r of level lt in global memory (right-hand side k at + k vol)
    T* z_out;                         // z of level lt in global memory
    int nlev;
    int nu;                           // smoothing sweeps before and after the coarse correction
    int ncoarse;                      // sweeps on a coarsest level of more than one column
    T omega;
};

// A z at level k of one column, zl = z at level k: the expression of
// k_mg_resid, fprev the vertical flux from below (0 at k = 0), replaced by
// the flux to level k + 1.
template <typename T>
__device__ __forceinline__ T tail_az(const OpView<T>& op, const Col<T>& col, const T* zl, int k, T& fprev) {
    const int pl = (int)op.plane;
    const T zc = zl[col.c];
    const T zu = k + 1 < op.nz ? zl[pl + col.c] : zc;
    const T f = ldro(op.wv + k) * (zc - zu);
    T h = col.me * (zc - zl[col.ce]);
    h = fma(col.mw, zc - zl[col.cw], h);
    h = fma(col.mn, zc - zl[col.cn], h);
    h = fma(col.ms, zc - zl[col.cs], h);
    const T az = fma(ldro(op.dk + k), h, col.area * fma(ldro(op.mass + k), zc, f - fprev));
    fprev = f;
    return az;
}

// The flux into level k0 of a column from below, as k_mg_resid starts a part.
template <typename T>
__device__ __forceinline__ T tail_flux_below(const OpView<T>& op, const Col<T>& col, const T* z, int k0) {
    const int pl = (int)op.plane;
    return k0 > 0 ? ldro(op.wv + k0 - 1) * (z[(k0 - 1) * pl + col.c] - z[k0 * pl + col.c]) : T(0);
}

// The cell loops of the tail deal (column, level range) units over the
// block: a column's levels are split into parts so that small levels still
// give every thread work; a thread builds its column's geometry once and
// walks the levels of its part.
struct TailUnits {
    int ncols, nz, parts, units;
    __device__ __forceinline__ TailUnits(int ncols_, int nz_) : ncols(ncols_), nz(nz_) {
        parts = max(1, min(nz, (TAIL_WARPS * 32) / ncols));
        units = ncols * parts;
    }
    __device__ __forceinline__ void unit(int u, int& c, int& k0, int& k1) const {
        const int part = u / ncols;
        c = u - part * ncols;
        k0 = part * nz / parts;
        k1 = (part + 1) * nz / parts;
    }
};

// Each kind of step below is one out-of-line function, called for every
// level: the cycle runs each step only a few times, and inlined copies at
// every call site would be fetched from beyond the instruction cache each
// time.  The level's view is passed by value (its table pointers cannot
// alias the step's stores).

// z = (ZMODE 2 ? z : 0) + om M^{-1} rin on one level: rows of 32 consecutive
// columns (flattened j n_x + i), each row taken by a group of nch warps (one
// per 16-level chunk), the rows dealt round-robin over the block's groups.
// Warps outside a group join the block barriers only.
template <typename T, int ZMODE>
__device__ __noinline__ void tail_smooth(const OpView<T> op, const T* rin, T* z, T om, T (*sh_y)[32],
                                         T (*sh_c)[32], T (*sh_z)[32], T (*sh_d)[32]) {
    const int lane = threadIdx.x, warp = threadIdx.y;
    const int nch = (op.nz + 15) / 16;
    const int G = TAIL_WARPS / nch;
    const bool in_grp = warp < G * nch;
    const int grp = in_grp ? warp / nch : 0;
    const int ch = in_grp ? warp - grp * nch : 0;
    const int w0 = in_grp ? grp * nch : warp;
    const int nch_c = in_grp ? nch : 1;
    const int ncols = (int)op.plane, nrow = (ncols + 31) / 32;
    const int rounds = (nrow + G - 1) / G;
    for (int rd = 0; rd < rounds; ++rd) {
        const int f = (rd * G + grp) * 32 + lane;
        int i = op.nx, j = 0;   // no column
        if (in_grp && f < ncols) {
            j = f / op.nx;
            i = f - j * op.nx;
        }
        const Col<T> col = make_col(op, i, j);
        Acc<T> sums[2];
        prec_chunked_body<T, 16, false, ZMODE>(op, col, lane, ch, nch_c, w0, const_cast<T*>(rin), rin, z, T(0), sums,
                                               sh_y, sh_c, sh_z, sh_d, nullptr, nullptr, 0, om);
    }
}

template <typename T>
__device__ __noinline__ void tail_resid(const OpView<T> op, const T* r, const T* z, T* t) {
    const TailUnits tu((int)op.plane, op.nz);
    const int pl = (int)op.plane;
    for (int u = threadIdx.y * 32 + threadIdx.x; u < tu.units; u += TAIL_WARPS * 32) {
        int c, k0, k1;
        tu.unit(u, c, k0, k1);
        const int j = c / op.nx;
        const Col<T> col = make_col(op, c - j * op.nx, j);
        T fprev = tail_flux_below(op, col, z, k0);
        for (int k = k0; k < k1; ++k) {
            const T az = tail_az(op, col, z + k * pl, k, fprev);
            t[k * pl + c] = r[k * pl + c] - az;
        }
    }
}

// rc = R (r - A z): the four fine residuals of a coarse cell summed in the
// order of k_mg_restrict.
template <typename T>
__device__ __noinline__ void tail_resid_restrict(const OpView<T> op, const T* r, const T* z, T* rc) {
    const int nxc = op.nx / 2, pl = (int)op.plane, plc = pl / 4;
    const TailUnits tu(plc, op.nz);
    for (int u = threadIdx.y * 32 + threadIdx.x; u < tu.units; u += TAIL_WARPS * 32) {
        int cc, k0, k1;
        tu.unit(u, cc, k0, k1);
        const int jc = cc / nxc, ic = cc - jc * nxc;
        const Col<T> c00 = make_col(op, 2 * ic, 2 * jc), c01 = make_col(op, 2 * ic + 1, 2 * jc);
        const Col<T> c10 = make_col(op, 2 * ic, 2 * jc + 1), c11 = make_col(op, 2 * ic + 1, 2 * jc + 1);
        T f00 = tail_flux_below(op, c00, z, k0), f01 = tail_flux_below(op, c01, z, k0);
        T f10 = tail_flux_below(op, c10, z, k0), f11 = tail_flux_below(op, c11, z, k0);
        for (int k = k0; k < k1; ++k) {
            const T* zl = z + k * pl;
            const T* rl = r + k * pl;
            const T t00 = rl[c00.c] - tail_az(op, c00, zl, k, f00);
            const T t01 = rl[c01.c] - tail_az(op, c01, zl, k, f01);
            const T t10 = rl[c10.c] - tail_az(op, c10, zl, k, f10);
            const T t11 = rl[c11.c] - tail_az(op, c11, zl, k, f11);
            rc[k * plc + cc] = ((t00 + t01) + t10) + t11;
        }
    }
}

// zf += P zc
template <typename T>
__device__ __noinline__ void tail_prolong(const OpView<T> op, const T* zc, T* zf) {
    const int nxc = op.nx / 2, pl = (int)op.plane, plc = pl / 4;
    const TailUnits tu(pl, op.nz);
    for (int u = threadIdx.y * 32 + threadIdx.x; u < tu.units; u += TAIL_WARPS * 32) {
        int c, k0, k1;
        tu.unit(u, c, k0, k1);
        const int j = c / op.nx, i = c - j * op.nx;
        const int cc = (j >> 1) * nxc + (i >> 1);
        for (int k = k0; k < k1; ++k) zf[k * pl + c] += zc[k * plc + cc];
    }
}

// Grid (nrhs), block (32, TAIL_WARPS), dynamic shared memory as laid out in
// a.off_*.  The sequence of steps is that of the launches it replaces.
template <typename T>
__global__ __launch_bounds__(TAIL_WARPS * 32) void k_mg_tail(const __grid_constant__ TailArgs<T> a,
                                                            const SolveState* __restrict__ st) {
    extern __shared__ __align__(16) unsigned char tail_smem[];
    __shared__ T sh_y[TAIL_WARPS][32], sh_c[TAIL_WARPS][32], sh_z[TAIL_WARPS][32], sh_d[TAIL_WARPS][32];
    const int rhs = blockIdx.x;
    if (st[rhs].done) return;
    T* sm = reinterpret_cast<T*>(tail_smem);
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int c = a.nlev - 1;
    T* const tt = sm + a.off_t;
    auto R = [&](int l) { return sm + a.off_r[l]; };
    auto Z = [&](int l) { return sm + a.off_z[l]; };
    auto smooth = [&](int l, const T* rin, T om, bool acc) {   // z = (acc ? z : 0) + om M^{-1} rin
        const OpView<T> op = a.op[l];
        if (acc)
            tail_smooth<T, 2>(op, rin, Z(l), om, sh_y, sh_c, sh_z, sh_d);
        else
            tail_smooth<T, 1>(op, rin, Z(l), om, sh_y, sh_c, sh_z, sh_d);
        __syncthreads();
    };
    auto resid = [&](int l) {                                  // t = r - A z
        const OpView<T> op = a.op[l];
        tail_resid(op, R(l), Z(l), tt);
        __syncthreads();
    };
    auto smooth_more = [&](int l) {                            // z += omega M^{-1} (r - A z)
        resid(l);
        smooth(l, tt, a.omega, true);
    };
    {
        const int v0 = (int)a.op[0].vol;
        const T* src = a.r_in + (long long)rhs * v0;
        T* dst = R(0);
        for (int u = tid; u < v0; u += TAIL_WARPS * 32) dst[u] = ldro(src + u);
        __syncthreads();
    }
    for (int l = 0; l < c; ++l) {
        smooth(l, R(l), a.omega, false);
        for (int k = 1; k < a.nu; ++k) smooth_more(l);
        const OpView<T> op = a.op[l];
        tail_resid_restrict(op, R(l), Z(l), R(l + 1));
        __syncthreads();
    }
    if (a.op[c].plane == 1) {   // one column: its block solve with one refinement step
        smooth(c, R(c), T(1), false);
        resid(c);
        smooth(c, tt, T(1), true);
    } else {
        smooth(c, R(c), a.omega, false);
        for (int k = 1; k < a.ncoarse; ++k) smooth_more(c);
    }
    for (int l = c - 1; l >= 0; --l) {
        const OpView<T> op = a.op[l];
        tail_prolong(op, Z(l + 1), Z(l));
        __syncthreads();
        for (int k = 0; k < a.nu; ++k) smooth_more(l);
    }
    {
        const int v0 = (int)a.op[0].vol;
        T* dst = a.z_out + (long long)rhs * v0;
        const T* src = Z(0);
        for (int u = tid; u < v0; u += TAIL_WARPS * 32) dst[u] = src[u];
    }
}

}  // namespace pcg
