// Single-reduction PCG (PCG_ALG_SINGLE_REDUCTION): one fused sweep per
// iteration.
//
// Section 4.3 of the paper points to the CG rearrangement of Chronopoulos and
// Gear (1989), which gathers an iteration's inner products into one
// reduction.  With u = M^{-1} r, w = A u, gamma = <r, u> and
// delta = <w, u>:
//   beta  = gamma / gamma_old                        (0 on the first step)
//   alpha = gamma / (delta - beta gamma / alpha_old)  (gamma / delta on the first step)
//   p = u + beta p,  s = w + beta s  (= A p),  x = x + alpha p,  r = r - alpha s.
// Algorithm 1 needs two grid-wide steps per iteration because the stencil
// needs z = M^{-1} r in the neighbouring columns.  Here a block solves the
// line systems of its tile of columns and of the ring of columns around it
// (r and s of a ring column are recomputed from the previous pass's r, s and
// w, bitwise as their owner computes them), so the stencil w = A u of its own
// columns needs nothing from other blocks of the same pass: one kernel and one
// reduction per iteration.  r, s and w are double-buffered (a ring column
// reads the previous pass's values while its owner writes the new ones); u,
// p and x are read and written by their owner only.
#pragma once
#include "kernels.cuh"

namespace pcg {

// A block's tile of own columns, per precision: in FP32 a warp covers 32
// columns of a row (whole 128-byte lines); in FP64 16 x 4, so that n_z x 108
// doubles of shared memory still allow n_z up to 256.
template <typename T>
struct SrTile {
    static constexpr int TX = sizeof(T) == 4 ? 32 : 16, TY = 4;
    static constexpr int HX = TX + 2, HY = TY + 2;   // with the ring around them
    static constexpr int NH = HX * HY;               // line solves per block: 204 (FP32), 108 (FP64)
    static constexpr int NT = 2 * TX * TY;           // threads: a ring slot each, then two per own column
    static_assert(NT >= NH, "phase 1 takes a ring slot per thread");
};
constexpr int SR_TY = 4;
constexpr int SR_MAX_NZ = 256;                        // u of the tile and its ring in shared memory
constexpr int SR_PB = 8;                              // levels whose loads are issued ahead

// Scalar step after the reduction of pass k: the stopping test on ||r||,
// then beta and alpha for pass k + 1.  x is current when the test fires, so
// alpha is set to 0 on every exit (the fix-up after the loop adds nothing).
__device__ __forceinline__ void sr_epilogue(SolveState* st, double rrv, double g, double d) {
    st->rr = rrv;
    st->kappa = g;
    st->sigma = d;
    st->pass += 1;
    if (!(isfinite(rrv) && isfinite(g) && isfinite(d)) || g < 0.0) {
        st->done = 1;
        st->status = 5;   // PCG_BREAKDOWN
        st->alpha = 0.0;
        return;
    }
    if (rrv == 0.0 || rrv < st->thresh2) {
        st->done = 1;
        st->status = 0;   // PCG_OK
        st->alpha = 0.0;
        return;
    }
    if (st->pass > st->maxit) {
        st->done = 1;
        st->status = 4;   // PCG_NOT_CONVERGED
        st->alpha = 0.0;
        return;
    }
    double beta = 0.0, den = d;
    if (st->pass > 1) {
        beta = g / st->kappa_old;
        den = d - beta * g / st->alpha;
    }
    if (!(den > 0.0) || !isfinite(den)) {
        st->done = 1;
        st->status = 5;   // PCG_BREAKDOWN
        st->alpha = 0.0;
        return;
    }
    st->beta = beta;
    st->alpha = g / den;
    st->kappa_old = g;
}

// One pass in precision T.  Grid (ceil(n_x/TX), ceil(n_y/4), nrhs), NT
// threads, n_z * NH values of T in dynamic shared memory (SrTile<T>).
//   Phase 1 (thread t < NH takes ring slot t): s' = w + beta s,
//   r' = r - alpha s', then the Thomas recurrences of Algorithm 3 into shared
//   memory, in FP64 in the c-form of the FP64 sweeps
//     y_k = r'_k + c_{k-1} y_{k-1},  t_k = y_k / D_k,  u_k = t_k + c_k u_{k+1},
//   in FP32 in the excess form of the FP32 sweeps (e = E/D, E = D - W)
//     y_k = (r'_k - e_{k-1} y_{k-1}) + y_{k-1},  u_k = u_{k+1} + (y_k - E_k u_{k+1}) / D_k;
//   gamma = <r', u'> = sum_k y_k^2 / D_k either way.  Own columns store r'
//   and s' and sum ||r'||^2 and gamma (in FP32 as plain sums over 8 levels,
//   both non-negative, added to the compensated accumulator).
//   Phase 2 (threads t and t + TX TY take the lower and upper half of own
//   column t): w' = A u' in flux form from shared memory (as k_apply), p' = u + beta p,
//   x += alpha p', delta += w' u' (compensated in FP32); stores u', p', x, w'.
// The last block to finish forms the scalars in FP64 (sr_epilogue).
template <typename T>
__global__ __launch_bounds__(SrTile<T>::NT) void k_sweep_sr(OpView<T> op, T* __restrict__ x, T* __restrict__ u,
                                                    T* __restrict__ p, const T* __restrict__ r_in,
                                                    T* __restrict__ r_out, const T* __restrict__ s_in,
                                                    T* __restrict__ s_out, const T* __restrict__ w_in,
                                                    T* __restrict__ w_out, SolveState* __restrict__ states,
                                                    double* __restrict__ partials, unsigned* __restrict__ counters,
                                                    int nblocks) {
    constexpr bool F64 = sizeof(T) == 8;
    constexpr int SR_TX = SrTile<T>::TX, SR_HX = SrTile<T>::HX, SR_NH = SrTile<T>::NH;
    extern __shared__ __align__(16) unsigned char sr_smem[];
    T* sh_u = reinterpret_cast<T*>(sr_smem);   // [n_z][NH]
    const int rhs = blockIdx.z;
    SolveState* st = states + rhs;
    if (st->done) return;
    const T alpha = (T)st->alpha, beta = (T)st->beta;
    const int nz = op.nz;
    const long long pl = op.plane, base = (long long)rhs * op.vol;
    const int i0 = blockIdx.x * SR_TX, j0 = blockIdx.y * SR_TY;
    const int tid = threadIdx.x;
    Acc<T> acc[3];   // ||r'||^2, gamma, delta over the block's own columns
    if (tid < SR_NH) {
        const int hx = tid % SR_HX, hy = tid / SR_HX;
        int i = i0 + hx - 1, j = j0 + hy - 1;
        const bool own = hx >= 1 && hx <= SR_TX && hy >= 1 && hy <= SR_TY && i < op.nx && j < op.ny;
        // ring columns wrap on a periodic axis and repeat the edge column on a
        // Neumann edge (the face weight there is 0), as make_col's neighbours do
        i = ((i % op.nx) + op.nx) % op.nx;
        j = op.periodic_y ? ((j % op.ny) + op.ny) % op.ny : min(max(j, 0), op.ny - 1);
        const long long c = (long long)j * op.nx + i;
        const int cls = op.cls_mode == 0 ? 0 : (op.cls_mode == 1 ? j : (int)c);
        const long long fs = op.ncls;
        const T* fg = op.fg + cls;
        const T* fx = (F64 ? op.fc : op.fe) + cls;   // c = W/D (FP64) or E = D - W (FP32)
        const long long o0 = base + c;
        // the loads of the next SR_PB levels are issued before the current SR_PB are computed
        T ra[SR_PB], sa[SR_PB], wa[SR_PB];
        auto fetch = [&](int kb, T(&vr)[SR_PB], T(&vs)[SR_PB], T(&vw)[SR_PB]) {
#pragma unroll
            for (int t = 0; t < SR_PB; ++t) {
                const int k = kb + t;
                if (k < nz) {
                    const long long o = o0 + (long long)k * pl;
                    vr[t] = r_in[o];
                    vs[t] = s_in[o];
                    vw[t] = w_in[o];
                }
            }
        };
        fetch(0, ra, sa, wa);
        T y = T(0), cprev = T(0);   // cprev: c_{k-1} (FP64) or e_{k-1} = E_{k-1} / D_{k-1} (FP32)
        for (int kb = 0; kb < nz; kb += SR_PB) {
            T rx[SR_PB], sx[SR_PB], wx[SR_PB];
            fetch(kb + SR_PB, rx, sx, wx);
            T rr_chunk = T(0), g_chunk = T(0);
#pragma unroll
            for (int t = 0; t < SR_PB; ++t) {
                const int k = kb + t;
                if (k < nz) {
                    const long long o = o0 + (long long)k * pl;
                    const T sn = fma(beta, sa[t], wa[t]);
                    const T rn = fma(-alpha, sn, ra[t]);
                    const T gk = ldro(fg + k * fs);
                    if constexpr (F64) {
                        y = fma(cprev, y, rn);
                        const T tk = gk * y;
                        if (own) {
                            acc[0].add_prod(rn, rn);
                            acc[1].add_prod(tk, y);
                        }
                        sh_u[k * SR_NH + tid] = tk;
                        cprev = ldro(fx + k * fs);
                    } else {
                        y = fma(-cprev, y, rn) + y;
                        rr_chunk = fma(rn, rn, rr_chunk);
                        g_chunk = fma(gk * y, y, g_chunk);
                        sh_u[k * SR_NH + tid] = y;
                        cprev = ldro(fx + k * fs) * gk;
                    }
                    if (own) {
                        s_out[o] = sn;
                        r_out[o] = rn;
                    }
                }
            }
            if constexpr (!F64) {
                if (own) {
                    acc[0].add(rr_chunk);
                    acc[1].add(g_chunk);
                }
            }
#pragma unroll
            for (int t = 0; t < SR_PB; ++t) {
                ra[t] = rx[t];
                sa[t] = sx[t];
                wa[t] = wx[t];
            }
        }
        T un = T(0);
        for (int k = nz - 1; k >= 0; --k) {
            T* sk = sh_u + k * SR_NH + tid;
            if constexpr (F64) un = fma(ldro(fx + k * fs), un, *sk);
            else un = fma(ldro(fg + k * fs), fma(-ldro(fx + k * fs), un, *sk), un);
            *sk = un;
        }
    }
    __syncthreads();
    {
        // two threads per own column, each over half of its levels (the flux
        // from below is recomputed at the split, with the same operands)
        const int oc = tid % (SR_TX * SR_TY), half = tid / (SR_TX * SR_TY);
        const int tx = oc % SR_TX, ty = oc / SR_TX;
        const Col<T> col = make_col(op, i0 + tx, j0 + ty);
        const int k0 = half * (nz / 2), k1 = half ? nz : nz / 2;
        if (col.valid && k0 < k1) {
            const int sc = (ty + 1) * SR_HX + tx + 1;
            const long long o0 = base + col.c;
            T pa[SR_PB], ua[SR_PB], xa[SR_PB];
            auto fetch = [&](int kb, T(&vp)[SR_PB], T(&vu)[SR_PB], T(&vx)[SR_PB]) {
#pragma unroll
                for (int t = 0; t < SR_PB; ++t) {
                    const int k = kb + t;
                    if (k < k1) {
                        const long long o = o0 + (long long)k * pl;
                        vp[t] = p[o];
                        vu[t] = u[o];
                        vx[t] = x[o];
                    }
                }
            };
            fetch(k0, pa, ua, xa);
            T zc = sh_u[k0 * SR_NH + sc];
            T fprev = k0 > 0 ? ldro(op.wv + k0 - 1) * (sh_u[(k0 - 1) * SR_NH + sc] - zc) : T(0);
            for (int kb = k0; kb < k1; kb += SR_PB) {
                T px[SR_PB], ux[SR_PB], xx[SR_PB];
                fetch(kb + SR_PB, px, ux, xx);
#pragma unroll
                for (int t = 0; t < SR_PB; ++t) {
                    const int k = kb + t;
                    if (k < k1) {
                        const T* sl = sh_u + k * SR_NH;
                        const T zu = (k + 1 < nz) ? sl[SR_NH + sc] : zc;
                        const T f = ldro(op.wv + k) * (zc - zu);
                        T h = col.me * (zc - sl[sc + 1]);
                        h = fma(col.mw, zc - sl[sc - 1], h);
                        h = fma(col.mn, zc - sl[sc + SR_HX], h);
                        h = fma(col.ms, zc - sl[sc - SR_HX], h);
                        const T wn = fma(ldro(op.dk + k), h, col.area * fma(ldro(op.mass + k), zc, f - fprev));
                        const long long o = o0 + (long long)k * pl;
                        const T pn = fma(beta, pa[t], ua[t]);
                        x[o] = fma(alpha, pn, xa[t]);
                        p[o] = pn;
                        u[o] = zc;
                        w_out[o] = wn;
                        acc[2].add_prod(wn, zc);
                        fprev = f;
                        zc = zu;
                    }
                }
#pragma unroll
                for (int t = 0; t < SR_PB; ++t) {
                    pa[t] = px[t];
                    ua[t] = ux[t];
                    xa[t] = xx[t];
                }
            }
        }
    }
    double v[3];
    if (grid_sum_acc<3>(acc, partials + (long long)rhs * nblocks * 3, counters + rhs, nblocks, bid2(), v))
        sr_epilogue(st, v[0], v[1], v[2]);
}

}  // namespace pcg
