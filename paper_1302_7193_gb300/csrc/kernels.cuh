// Device kernels of the matrix-free line-preconditioned CG solver (sm_103a).
//
// Data layout: every vector is [nrhs][n_z][n_y][n_x] with x fastest, so a
// vertical level is one contiguous horizontal plane and a warp of threads
// that own neighbouring columns reads 32 consecutive values per level
// (the coalescing argument of Section 6.1, Eq. (MemoryMappingCUDAC)).
//
// Parallelisation: one thread per vertical column for the kernels that carry
// the vertical recurrence of the Thomas algorithm (Section 6.1: the line
// solve is sequential in the vertical); threads are grouped in 32 x 4 tiles
// of columns.  The k-loop keeps the column's current, next and previous
// values and the running vertical flux in registers.
//
// Operator (Section 3.1, Eq. (TridiagonalMatrix), Section 4.2 stencil) in
// flux form:
//   (A z)_{ijk} = |T_j| ( m_k z_k + F_k - F_{k-1} ) + d_k sum_f mu_f (z_k - z_f),
//   F_k = w_k (z_k - z_{k+1})   (w_{n_z-1} = 0: Neumann top; F_{-1} = 0: Neumann bottom).
// Each flux is computed once and enters rows k and k+1 with opposite signs,
// and every neighbour enters through an exact difference, so A 1 = |T| m
// exactly and near-constant vectors lose no precision to cancellation.
//
// Preconditioner (Section 4.2, Eq. (MatrixFreeTridiagonalSystem)): per
// column M = L D L^T with pivots D_k = W_k + E_k (W_k = |T| w_k the coupling
// to level k+1, E_k >= 0 the pivot's excess over it).  With precomputed
// g_k = 1/D_k and E_k the two Thomas sweeps read
//   forward:  y_k = (r_k - e_{k-1} y_{k-1}) + y_{k-1},   e = E g  (= 1 - W/D),
//   backward: z_k = z_{k+1} + g_k (y_k - E_k z_{k+1}),
// which is the textbook recurrence y_k = r_k + (W/D) y_{k-1},
// z_k = (y_k + W_k z_{k+1})/D_k written so that the small excesses are never
// added to or subtracted from the large couplings: at strong anisotropy W/D
// rounds to 1 in FP32 and the column's near-constant mode would be lost.
// <r, M^{-1} r> = sum_k g_k y_k^2 is accumulated in the forward sweep.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pcg {

constexpr int BX = 32;
constexpr int BY = 4;
constexpr int NT = BX * BY;

// Per right-hand-side scalar state of one PCG solve (Algorithm 1).
struct SolveState {
    double alpha;       // step length of the last SpMV sweep (0 before the first)
    double beta;        // kappa / kappa_old of the last preconditioner sweep
    double kappa_old;   // <r, z> of the previous pass (1 before the first)
    double sigma;       // <p, q> of the last SpMV sweep
    double rr;          // <r, r> of the last preconditioner sweep
    double kappa;       // <r, z> of the last preconditioner sweep
    double bnorm2;      // <b, b>
    double thresh2;     // stop when rr < thresh2 (= tol^2 <b, b>)
    double tol2;        // tol^2 as requested
    double rr_true;     // <b - A x, b - A x> after the solve
    double rsum;        // sum_i (b - A x)_i (refinement: constant-mode projection)
    double coarse;      // constant added to x by the refinement's coarse correction
    double rr_emit;     // <r', r'> of the inner right-hand side r' = b - A x - coarse A 1
    double floor2;      // sum_i ulp(x_i)^2/12 ||A e_i||^2: expected ||A (fl(x) - x)||^2 of rounding x to FP64
    int done;           // 1 once the solve of this rhs has stopped
    int status;         // pcg_status of this rhs
    int pass;           // preconditioner sweeps completed
    int maxit;          // iteration cap
    int zero_rhs;       // b == 0: the solution is 0
    int pad_;
};

// Read-only view of the operator tables in precision T.
template <typename T>
struct OpView {
    int nx, ny, nz;
    long long plane;            // nx * ny
    long long vol;              // plane * nz (one right-hand side)
    const T* mass;              // [nz] zero-order term per unit area
    const T* wv;                // [nz] vertical coupling per unit area between k and k+1 (0 at the top)
    const T* dk;                // [nz] weight of the horizontal couplings per level
    const T* area;              // [ny] |T_j|, or [ny][nx] |T_ij| when area_percol
    const T* mue;               // [ny][nx] east-face weight
    const T* mun;               // [ny][nx] north-face weight (0 on a Neumann edge)
    int periodic_y;
    const T* fg;                // [nz][ncls] 1 / D_k
    const T* fe;                // [nz][ncls] E_k = D_k - W_k
    const T* fc;                // [nz][ncls] c_k = W_k / D_k (FP64 sweeps only; may be null in FP32 views)
    int cls_mode;               // 0: one factor set; 1: per row j; 2: per column
    int ncls;
    int area_percol;            // 1: area indexed by column (cubed-sphere panel)
    const T* amass;             // [rows][nz] |T| a_k with the area folded in, or null (area per column)
    const T* awv;               // [rows][nz] |T| w_k
    int arow_step;              // 0: one folded row (uniform area); 1: one per grid row j
};

// Per-thread accumulators: plain FP64, or compensated FP32 (exact product
// error by FMA, TwoSum accumulation) converted to FP64 at the end.
template <typename T> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ void add(double a) { s += a; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        float p = a * b;
        float pe = fmaf(a, b, -p);
        float t = s + p;
        float bp = t - s;
        float e = (s - (t - bp)) + (p - bp);
        s = t;
        c += e + pe;
    }
    // add an exact-enough partial sum (TwoSum, error kept in c)
    __device__ __forceinline__ void add(float a) {
        const float t = s + a;
        const float bp = t - s;
        c += (s - (t - bp)) + (a - bp);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <typename T>
__device__ __forceinline__ T ldro(const T* p) { return __ldg(p); }

// Geometry of one column: neighbour offsets within a plane and face weights.
template <typename T>
struct Col {
    long long c, ce, cw, cn, cs;
    T area, me, mw, mn, ms;
    int j;                      // grid row
    int cls;
    bool valid;
};

template <typename T>
__device__ __forceinline__ Col<T> make_col(const OpView<T>& op, int i, int j) {
    Col<T> col;
    col.valid = (i < op.nx) && (j < op.ny);
    const int ii = col.valid ? i : 0;
    const int jj = col.valid ? j : 0;
    const int ie = (ii + 1 == op.nx) ? 0 : ii + 1;
    const int iw = (ii == 0) ? op.nx - 1 : ii - 1;
    int jn, js;
    if (op.periodic_y) {
        jn = (jj + 1 == op.ny) ? 0 : jj + 1;
        js = (jj == 0) ? op.ny - 1 : jj - 1;
    } else {
        jn = (jj + 1 == op.ny) ? jj : jj + 1;   // weight is 0 there
        js = (jj == 0) ? jj : jj - 1;
    }
    const long long nx = op.nx;
    col.c = (long long)jj * nx + ii;
    col.ce = (long long)jj * nx + ie;
    col.cw = (long long)jj * nx + iw;
    col.cn = (long long)jn * nx + ii;
    col.cs = (long long)js * nx + ii;
    col.area = ldro(op.area + (op.area_percol ? col.c : (long long)jj));
    col.me = ldro(op.mue + col.c);
    col.mw = ldro(op.mue + col.cw);
    col.mn = ldro(op.mun + col.c);
    col.ms = (op.periodic_y || jj > 0) ? ldro(op.mun + col.cs) : T(0);
    col.cls = op.cls_mode == 0 ? 0 : (op.cls_mode == 1 ? jj : (int)col.c);
    col.j = jj;
    return col;
}

// Horizontal part sum_f mu_f (z_c - z_f) at one level; zl points at the plane.
template <typename T>
__device__ __forceinline__ T horiz(const Col<T>& col, const T* __restrict__ zl, T zc) {
    T a = col.me * (zc - ldro(zl + col.ce));
    a = fma(col.mw, zc - ldro(zl + col.cw), a);
    a = fma(col.mn, zc - ldro(zl + col.cn), a);
    a = fma(col.ms, zc - ldro(zl + col.cs), a);
    return a;
}

// ---------------------------------------------------------------------------
// Block / grid reductions with a deterministic order.
// ---------------------------------------------------------------------------
constexpr int MAXW = 8;   // blocks of at most 256 threads

template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double (*sh)[MAXW]) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
    for (int n = 0; n < N; ++n) {
        double a = v[n];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if ((tid & 31) == 0) sh[n][tid >> 5] = a;
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int n = 0; n < N; ++n) {
            double a = 0.0;
            for (int w = 0; w < nw; ++w) a += sh[n][w];
            v[n] = a;
        }
    }
}

// Each block stores its N partial sums at index `bid`; the last block to
// arrive sums all partials of its right-hand side in block order and returns
// true on thread 0 (with the totals in v).  Other threads return false.
template <int N>
__device__ __forceinline__ bool grid_sum(double (&v)[N], double* partials, unsigned* counter, int nblocks, int bid) {
    __shared__ double sh[N][MAXW];
    __shared__ bool am_last;
    __shared__ double tot[N][MAXW];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    block_sum<N>(v, sh);
    if (tid == 0) {
#pragma unroll
        for (int n = 0; n < N; ++n) partials[(long long)bid * N + n] = v[n];
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        am_last = (prev == (unsigned)nblocks - 1u);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    double acc[N];
#pragma unroll
    for (int n = 0; n < N; ++n) acc[n] = 0.0;
    for (int b = tid; b < nblocks; b += nthr) {
#pragma unroll
        for (int n = 0; n < N; ++n) acc[n] += __ldcg(partials + (long long)b * N + n);
    }
    __syncthreads();
    block_sum<N>(acc, tot);
    if (tid == 0) {
#pragma unroll
        for (int n = 0; n < N; ++n) v[n] = acc[n];
        *counter = 0u;
    }
    return tid == 0;
}

__device__ __forceinline__ int bid2() { return blockIdx.y * gridDim.x + blockIdx.x; }

// Block-level sum of per-thread accumulators, then the cross-block FP64 sum
// of grid_sum.  FP32 accumulators are combined as compensated (sum, error)
// pairs with TwoSum so that FP32 kernels issue no FP64 instruction until one
// conversion per block (the FP64 pipe of this part is 1/64 of the FP32 rate).
__device__ __forceinline__ void pair_add(float& s, float& c, float s2, float c2) {
    const float t = s + s2;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (s2 - bp);
    s = t;
    c = c + c2 + e;
}

template <int N>
__device__ __forceinline__ bool grid_sum_acc(Acc<float> (&a)[N], double* partials, unsigned* counter, int nblocks,
                                             int bid, double (&out)[N]) {
    __shared__ float shs[N][MAXW], shc[N][MAXW];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
    for (int n = 0; n < N; ++n) {
        float s = a[n].s, c = a[n].c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, s, o);
            const float c2 = __shfl_down_sync(0xffffffffu, c, o);
            pair_add(s, c, s2, c2);
        }
        if ((tid & 31) == 0) {
            shs[n][tid >> 5] = s;
            shc[n][tid >> 5] = c;
        }
    }
    __syncthreads();
    double v[N];
#pragma unroll
    for (int n = 0; n < N; ++n) v[n] = 0.0;
    if (tid == 0) {
#pragma unroll
        for (int n = 0; n < N; ++n) {
            float s = shs[n][0], c = shc[n][0];
            for (int w = 1; w < nw; ++w) pair_add(s, c, shs[n][w], shc[n][w]);
            v[n] = (double)s + (double)c;
        }
    }
    // cross-block part (only thread 0's v is meaningful, as in grid_sum)
    __shared__ bool am_last;
    __shared__ double tot[N][MAXW];
    const int nthr = blockDim.x * blockDim.y;
    if (tid == 0) {
#pragma unroll
        for (int n = 0; n < N; ++n) partials[(long long)bid * N + n] = v[n];
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        am_last = (prev == (unsigned)nblocks - 1u);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    double acc[N];
#pragma unroll
    for (int n = 0; n < N; ++n) acc[n] = 0.0;
    for (int b = tid; b < nblocks; b += nthr) {
#pragma unroll
        for (int n = 0; n < N; ++n) acc[n] += __ldcg(partials + (long long)b * N + n);
    }
    block_sum<N>(acc, tot);
    if (tid == 0) {
#pragma unroll
        for (int n = 0; n < N; ++n) out[n] = acc[n];
        *counter = 0u;
    }
    return tid == 0;
}

// The block-level part of grid_sum_acc alone: the block's compensated FP32
// sums merged in the same order, converted to FP64 and written by thread 0
// to dst[0 .. N-1].  Holds one block barrier; the cross-block sum is left to
// a later kernel (the served batch's per-request scalar step).
template <int N>
__device__ __forceinline__ void block_partials(Acc<float> (&a)[N], double* dst) {
    __shared__ float shs[N][MAXW], shc[N][MAXW];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
    for (int n = 0; n < N; ++n) {
        float s = a[n].s, c = a[n].c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, s, o);
            const float c2 = __shfl_down_sync(0xffffffffu, c, o);
            pair_add(s, c, s2, c2);
        }
        if ((tid & 31) == 0) {
            shs[n][tid >> 5] = s;
            shc[n][tid >> 5] = c;
        }
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int n = 0; n < N; ++n) {
            float s = shs[n][0], c = shc[n][0];
            for (int w = 1; w < nw; ++w) pair_add(s, c, shs[n][w], shc[n][w]);
            dst[n] = (double)s + (double)c;
        }
    }
}

template <int N>
__device__ __forceinline__ bool grid_sum_acc(Acc<double> (&a)[N], double* partials, unsigned* counter, int nblocks,
                                             int bid, double (&out)[N]) {
#pragma unroll
    for (int n = 0; n < N; ++n) out[n] = a[n].value();
    return grid_sum<N>(out, partials, counter, nblocks, bid);
}


// Scalar steps of Algorithm 1 after the preconditioner sweep (lines 3-4):
// the stopping test on the updated residual and beta = kappa / kappa_old.
__device__ __forceinline__ void prec_epilogue(SolveState* st, double rrv, double kv) {
    st->rr = rrv;
    st->kappa = kv;
    st->pass += 1;
    if (!(isfinite(rrv) && isfinite(kv)) || kv < 0.0) {
        st->done = 1;
        st->status = 5;   // PCG_BREAKDOWN
    } else if (rrv == 0.0 || rrv < st->thresh2) {
        st->done = 1;
        st->status = 0;   // PCG_OK
    } else if (st->pass > st->maxit) {
        st->done = 1;
        st->status = 4;   // PCG_NOT_CONVERGED
    } else {
        st->beta = kv / st->kappa_old;
        st->kappa_old = kv;
    }
}

// Scalar step after the SpMV sweep (line 6): alpha = kappa_old / sigma.
__device__ __forceinline__ void spmv_epilogue(SolveState* st, double s) {
    st->sigma = s;
    if (*(volatile int*)&st->status == 6) {   // a block's staged copies timed out (PCG_TIMEOUT)
        st->done = 1;
        st->alpha = 0.0;
        return;
    }
    if (!(s > 0.0) || !isfinite(s)) {
        st->done = 1;
        st->status = 5;   // PCG_BREAKDOWN
        st->alpha = 0.0;
    } else {
        st->alpha = st->kappa_old / s;
    }
}

// ---------------------------------------------------------------------------
// y = A x
// ---------------------------------------------------------------------------
template <typename T>
__global__ __launch_bounds__(NT) void k_apply(OpView<T> op, const T* __restrict__ x, T* __restrict__ y) {
    const Col<T> col = make_col(op, blockIdx.x * BX + threadIdx.x, blockIdx.y * BY + threadIdx.y);
    if (!col.valid) return;
    const long long base = (long long)blockIdx.z * op.vol;
    const T* __restrict__ xb = x + base;
    T* __restrict__ yb = y + base;
    T zc = xb[col.c];
    T fprev = T(0);
#pragma unroll 4
    for (int k = 0; k < op.nz; ++k) {
        const T* xl = xb + (long long)k * op.plane;
        const T zu = (k + 1 < op.nz) ? ldro(xl + op.plane + col.c) : zc;
        const T f = ldro(op.wv + k) * (zc - zu);
        const T hz = horiz(col, xl, zc);
        yb[(long long)k * op.plane + col.c] =
            fma(ldro(op.dk + k), hz, col.area * fma(ldro(op.mass + k), zc, f - fprev));
        fprev = f;
        zc = zu;
    }
}

// ---------------------------------------------------------------------------
// z = M^{-1} r (one Thomas solve per column)
// ---------------------------------------------------------------------------
template <typename T>
__global__ __launch_bounds__(NT) void k_precond(OpView<T> op, const T* __restrict__ r, T* __restrict__ z) {
    const Col<T> col = make_col(op, blockIdx.x * BX + threadIdx.x, blockIdx.y * BY + threadIdx.y);
    if (!col.valid) return;
    const long long base = (long long)blockIdx.z * op.vol;
    const T* rb = r + base;
    T* zb = z + base;
    const T* fg = op.fg + col.cls;
    const long long fs = op.ncls;
    if constexpr (sizeof(T) == 8) {
        // FP64: c form, as in prec_column
        const T* fc = op.fc + col.cls;
        T y = T(0), cprev = T(0);
#pragma unroll 4
        for (int k = 0; k < op.nz; ++k) {
            const long long o = (long long)k * op.plane + col.c;
            y = fma(cprev, y, rb[o]);
            zb[o] = ldro(fg + k * fs) * y;
            cprev = ldro(fc + k * fs);
        }
        T zn = T(0);
#pragma unroll 4
        for (int k = op.nz - 1; k >= 0; --k) {
            const long long o = (long long)k * op.plane + col.c;
            zn = fma(ldro(fc + k * fs), zn, zb[o]);
            zb[o] = zn;
        }
    } else {
        const T* fe = op.fe + col.cls;
        T y = T(0), eprev = T(0);
#pragma unroll 4
        for (int k = 0; k < op.nz; ++k) {
            y = fma(-eprev, y, rb[(long long)k * op.plane + col.c]) + y;
            zb[(long long)k * op.plane + col.c] = y;
            eprev = ldro(fe + k * fs) * ldro(fg + k * fs);
        }
        T zn = T(0);
#pragma unroll 4
        for (int k = op.nz - 1; k >= 0; --k) {
            const long long o = (long long)k * op.plane + col.c;
            zn = fma(ldro(fg + k * fs), fma(-ldro(fe + k * fs), zn, zb[o]), zn);
            zb[o] = zn;
        }
    }
}

// ---------------------------------------------------------------------------
// Preconditioner sweep of Algorithm 1 (Algorithm 3): r <- r - alpha q,
// <r, r>, z = M^{-1} r, kappa = <r, z>; the last block applies the stopping
// test and forms beta = kappa / kappa_old.
// ---------------------------------------------------------------------------
// One column of the preconditioner sweep; r, q, z point at the column's
// level-0 entry.
template <typename T, bool PIPE = false>
__device__ __forceinline__ void prec_column(const OpView<T>& op, const Col<T>& col, T* __restrict__ rb,
                                            const T* __restrict__ qb, T* __restrict__ zb, T alpha, Acc<T>& rr,
                                            Acc<T>& kap) {
    const T* fg = op.fg + col.cls;
    const long long fs = op.ncls;
    if constexpr (sizeof(T) == 8) {
        // FP64: the Thomas recurrences with the stored ratio c_k = W_k / D_k,
        //   y_k = r_k + c_{k-1} y_{k-1},  t_k = y_k / D_k,  kappa += t_k y_k,
        //   z_k = t_k + c_k z_{k+1},
        // six FP64 operations per unknown with the residual update and norm.
        // c_k is one rounding of the exact ratio, so the excess 1 - c_k keeps a
        // relative accuracy of 2^-53 / (1 - c_k), ample in FP64 (the FP32
        // sweeps below cannot afford it and carry E_k instead).
        if constexpr (!PIPE) {
            const T* fc = op.fc + col.cls;
            T y = T(0), cprev = T(0);
    #pragma unroll 4
            for (int k = 0; k < op.nz; ++k) {
                const long long o = (long long)k * op.plane;
                const T rn = fma(-alpha, qb[o], rb[o]);
                rb[o] = rn;
                rr.add_prod(rn, rn);
                y = fma(cprev, y, rn);
                const T t = ldro(fg + k * fs) * y;
                kap.add_prod(t, y);
                zb[o] = t;
                cprev = ldro(fc + k * fs);
            }
            T zn = T(0);
    #pragma unroll 4
            for (int k = op.nz - 1; k >= 0; --k) {
                const long long o = (long long)k * op.plane;
                zn = fma(ldro(fc + k * fs), zn, zb[o]);
                zb[o] = zn;
            }
        } else {
            // The loads of the next PB levels are issued before the current PB
            // levels are computed and stored (the stores go to the same arrays,
            // so the compiler cannot hoist the loads over them by itself).
            constexpr int PB = 8;
            const T* fc = op.fc + col.cls;
            const long long pl = op.plane;
            const int nz = op.nz;
            T y = T(0), cprev = T(0);
            T ra[PB], qa[PB];
    #pragma unroll
            for (int t = 0; t < PB; ++t) {
                ra[t] = t < nz ? rb[t * pl] : T(0);
                qa[t] = t < nz ? qb[t * pl] : T(0);
            }
            for (int k0 = 0; k0 < nz; k0 += PB) {
                T rn_[PB], qn_[PB];
    #pragma unroll
                for (int t = 0; t < PB; ++t) {
                    const int k = k0 + PB + t;
                    rn_[t] = k < nz ? rb[k * pl] : T(0);
                    qn_[t] = k < nz ? qb[k * pl] : T(0);
                }
    #pragma unroll
                for (int t = 0; t < PB; ++t) {
                    const int k = k0 + t;
                    if (k < nz) {
                        const T rn = fma(-alpha, qa[t], ra[t]);
                        rb[k * pl] = rn;
                        rr.add_prod(rn, rn);
                        y = fma(cprev, y, rn);
                        const T tk = ldro(fg + k * fs) * y;
                        kap.add_prod(tk, y);
                        zb[k * pl] = tk;
                        cprev = ldro(fc + k * fs);
                    }
                }
    #pragma unroll
                for (int t = 0; t < PB; ++t) {
                    ra[t] = rn_[t];
                    qa[t] = qn_[t];
                }
            }
            // backward: z_k = t_k + c_k z_{k+1}, with the t of the next PB levels
            // (below) loaded before the current ones are overwritten
            T zn = T(0);
            T ta[PB];
            const int kt = nz - 1;
    #pragma unroll
            for (int t = 0; t < PB; ++t) ta[t] = kt - t >= 0 ? zb[(kt - t) * pl] : T(0);
            for (int k0 = kt; k0 >= 0; k0 -= PB) {
                T tn[PB];
    #pragma unroll
                for (int t = 0; t < PB; ++t) {
                    const int k = k0 - PB - t;
                    tn[t] = k >= 0 ? zb[k * pl] : T(0);
                }
    #pragma unroll
                for (int t = 0; t < PB; ++t) {
                    const int k = k0 - t;
                    if (k >= 0) {
                        zn = fma(ldro(fc + k * fs), zn, ta[t]);
                        zb[k * pl] = zn;
                    }
                }
    #pragma unroll
                for (int t = 0; t < PB; ++t) ta[t] = tn[t];
            }
        }
    } else {
        const T* fe = op.fe + col.cls;
        T y = T(0), eprev = T(0);
#pragma unroll 4
        for (int k = 0; k < op.nz; ++k) {
            const long long o = (long long)k * op.plane;
            const T rn = fma(-alpha, qb[o], rb[o]);
            rb[o] = rn;
            rr.add_prod(rn, rn);
            y = fma(-eprev, y, rn) + y;
            zb[o] = y;
            const T g = ldro(fg + k * fs);
            kap.add_prod(g * y, y);
            eprev = ldro(fe + k * fs) * g;
        }
        T zn = T(0);
#pragma unroll 4
        for (int k = op.nz - 1; k >= 0; --k) {
            const long long o = (long long)k * op.plane;
            zn = fma(ldro(fg + k * fs), fma(-ldro(fe + k * fs), zn, zb[o]), zn);
            zb[o] = zn;
        }
    }
}

// PIPE: FP64 Thomas with the next levels' loads issued ahead (for grids with
// few columns, where occupancy cannot hide the load latency)
template <typename T, bool PIPE = false>
__global__ __launch_bounds__(NT) void k_sweep_prec(OpView<T> op, T* __restrict__ r, const T* __restrict__ q,
                                                   T* __restrict__ z, SolveState* __restrict__ states,
                                                   double* __restrict__ partials, unsigned* __restrict__ counters,
                                                   int nblocks) {
    const int rhs = blockIdx.z;
    SolveState* st = states + rhs;
    if (st->done) return;
    const T alpha = (T)st->alpha;
    const Col<T> col = make_col(op, blockIdx.x * BX + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
    Acc<T> acc[2];
    if (col.valid) {
        const long long base = (long long)rhs * op.vol + col.c;
        prec_column<T, PIPE>(op, col, r + base, q + base, z + base, alpha, acc[0], acc[1]);
    }
    double v[2];
    if (grid_sum_acc<2>(acc, partials + (long long)rhs * nblocks * 2, counters + rhs, nblocks, bid2(), v))
        prec_epilogue(st, v[0], v[1]);
}

// ---------------------------------------------------------------------------
// SpMV sweep of Algorithm 1 (Algorithm 2): u <- u + alpha p, p <- z + beta p,
// q <- A z + beta q, sigma = <p, q>; the last block forms alpha = kappa_old/sigma.
// ---------------------------------------------------------------------------
// One column of the SpMV sweep; u, p, q point at the column's level-0
// entry, zb at level 0 of the right-hand side's z (the stencil reads
// neighbouring columns).
template <typename T, bool FOLD = false, bool PIPE = false>
__device__ __forceinline__ void spmv_column(const OpView<T>& op, const Col<T>& col, T* __restrict__ ub,
                                            T* __restrict__ pb, T* __restrict__ qb, const T* __restrict__ zb,
                                            T alpha, T beta, Acc<T>& sig, int k0 = 0, int k1 = -1) {
    // FOLD: the area is folded into the level tables (|T| a_k, |T| w_k per
    // row), one multiplication fewer per unknown for uniform or per-row areas.
    // Levels k0 .. k1-1 (default all); the flux into level k0 from below is
    // recomputed from z at k0-1.
    if (k1 < 0) k1 = op.nz;
    const T* am = FOLD ? op.amass + (op.arow_step ? (long long)col.j * op.nz : 0LL) : op.mass;
    const T* aw = FOLD ? op.awv + (op.arow_step ? (long long)col.j * op.nz : 0LL) : op.wv;
    T zc = zb[(long long)k0 * op.plane + col.c];
    T fprev = k0 > 0 ? ldro(aw + k0 - 1) * (zb[(long long)(k0 - 1) * op.plane + col.c] - zc) : T(0);
    // one level: uk, pk, qk are the loaded u, p, q at level k
    auto level = [&](int k, T uk, T pk, T qk) {
        const long long o = (long long)k * op.plane;
        const T* zl = zb + o;
        const T zu = (k + 1 < op.nz) ? ldro(zl + op.plane + col.c) : zc;
        ub[o] = fma(alpha, pk, uk);
        const T pn = fma(beta, pk, zc);
        pb[o] = pn;
        const T f = ldro(aw + k) * (zc - zu);
        const T hz = horiz(col, zl, zc);
        const T vz = fma(ldro(am + k), zc, f - fprev);
        const T az = fma(ldro(op.dk + k), hz, FOLD ? vz : col.area * vz);
        const T qn = fma(beta, qk, az);
        qb[o] = qn;
        sig.add_prod(pn, qn);
        fprev = f;
        zc = zu;
    };
    if constexpr (!PIPE) {
#pragma unroll 4
        for (int k = k0; k < k1; ++k) {
            const long long o = (long long)k * op.plane;
            level(k, ub[o], pb[o], qb[o]);
        }
    } else {
        // u, p, q of the next PB levels are loaded before the current PB levels
        // are stored (same arrays: the compiler cannot reorder them itself)
        constexpr int PB = 4;
        const long long pl = op.plane;
        T ua[PB], pa[PB], qa[PB];
#pragma unroll
        for (int t = 0; t < PB; ++t) {
            const int k = k0 + t;
            ua[t] = k < k1 ? ub[k * pl] : T(0);
            pa[t] = k < k1 ? pb[k * pl] : T(0);
            qa[t] = k < k1 ? qb[k * pl] : T(0);
        }
        for (int kb = k0; kb < k1; kb += PB) {
            T un[PB], pn[PB], qn[PB];
#pragma unroll
            for (int t = 0; t < PB; ++t) {
                const int k = kb + PB + t;
                un[t] = k < k1 ? ub[k * pl] : T(0);
                pn[t] = k < k1 ? pb[k * pl] : T(0);
                qn[t] = k < k1 ? qb[k * pl] : T(0);
            }
#pragma unroll
            for (int t = 0; t < PB; ++t)
                if (kb + t < k1) level(kb + t, ua[t], pa[t], qa[t]);
#pragma unroll
            for (int t = 0; t < PB; ++t) {
                ua[t] = un[t];
                pa[t] = pn[t];
                qa[t] = qn[t];
            }
        }
    }
}

// blockIdx.z = rhs * ksplit + part: part takes levels [part n_z / ksplit,
// (part + 1) n_z / ksplit) of every column of the tile (more, shorter threads
// that spread evenly over the SMs).
template <typename T, bool PIPE = false>
__global__ __launch_bounds__(NT) void k_sweep_spmv(OpView<T> op, T* __restrict__ u, T* __restrict__ p,
                                                   T* __restrict__ q, const T* __restrict__ z,
                                                   SolveState* __restrict__ states, double* __restrict__ partials,
                                                   unsigned* __restrict__ counters, int nblocks, int ksplit = 1) {
    const int rhs = blockIdx.z / ksplit;
    const int part = blockIdx.z - rhs * ksplit;
    const int k0 = (int)((long long)part * op.nz / ksplit), k1 = (int)((long long)(part + 1) * op.nz / ksplit);
    SolveState* st = states + rhs;
    if (st->done) return;
    const T alpha = (T)st->alpha;
    const T beta = (T)st->beta;
    const Col<T> col = make_col(op, blockIdx.x * BX + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
    Acc<T> sig[1];
    if (col.valid) {
        const long long base = (long long)rhs * op.vol;
        if (sizeof(T) == 8 && op.amass)
            spmv_column<T, true, PIPE>(op, col, u + base + col.c, p + base + col.c, q + base + col.c, z + base, alpha,
                                       beta, sig[0], k0, k1);
        else
            spmv_column<T, false, PIPE>(op, col, u + base + col.c, p + base + col.c, q + base + col.c, z + base, alpha,
                                        beta, sig[0], k0, k1);
    }
    double v[1];
    const int bid = (part * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (grid_sum_acc<1>(sig, partials + (long long)rhs * nblocks * 2, counters + rhs, nblocks, bid, v))
        spmv_epilogue(st, v[0]);
}

// ---------------------------------------------------------------------------
// The same two sweeps with each column split into chunks of LZ levels.
//
// One thread per (column, chunk) multiplies the number of threads by
// n_z / LZ, and every load of a chunk is issued before any arithmetic (into
// registers, and for the stencil's neighbours into a shared-memory tile), so
// many more bytes are in flight per SM than with one thread per column.
// The Thomas sweeps are linear recurrences with known coefficients, so a
// chunk solves its part with zero carry-in and is corrected afterwards:
//   forward   y_k = yl_k + P_k Y,   P_k = prod_{j=k0..k} (W_{j-1}/D_{j-1}),
//   backward  z_k = zl_k + Q_k Z,   Q_k = prod_{j=k..k1-1} (W_j/D_j),
// where Y (Z) is the true value just below (above) the chunk, obtained by a
// scan over the chunks of the column in shared memory.  The products are
// carried as C = 1 - P and D = 1 - Q built as C + e (1 - C) with
// e = E/D_pivot, so no quantity close to 1 is subtracted from 1: this is the
// excess form of the sweeps above, reassociated.
// Preconditioner sweep: block = 32 columns of one row x (n_z/LZ) chunks.
// ---------------------------------------------------------------------------
// One (column, chunk) of the chunked preconditioner sweep.  The chunks of a
// column are the warps w0 .. w0 + nch - 1 of the block (lane = column);
// r, q, z point at level 0 of the right-hand side.  The chunk's r and q are
// read from rsrc / qsrc (level t of the chunk at t * sstride; null: from r
// and q themselves); STORE_R = false leaves r unwritten.  Every thread of
// the block must call this (it holds two block barriers); threads with
// col.valid false take part in the barriers only.
// ZMODE: how the solution m = M^{-1} (r - alpha q) is stored: z = m (0),
// z = omega m (1) or z += omega m (2, a damped smoothing step).
template <typename T, int LZ, bool STORE_R = true, int ZMODE = 0>
__device__ __forceinline__ void prec_chunked_body(const OpView<T>& op, const Col<T>& col, int lane, int ch, int nch,
                                                  int w0, T* __restrict__ r, const T* __restrict__ q,
                                                  T* __restrict__ z, T alpha, Acc<T> (&acc)[2], T (*sh_y)[32],
                                                  T (*sh_c)[32], T (*sh_z)[32], T (*sh_d)[32],
                                                  const T* rsrc = nullptr, const T* qsrc = nullptr,
                                                  int sstride = 0, T omega = T(1)) {
    const int k0 = ch * LZ;
    const int kn = min(LZ, op.nz - k0);          // levels in this chunk (<= 0: none)
    const bool act = col.valid && kn > 0;
    const bool full = act && kn == LZ;
    const long long base = col.c;
    T* rb = r + base + (long long)k0 * op.plane;
    const T* qb = q + base + (long long)k0 * op.plane;
    T* zb = z + base + (long long)k0 * op.plane;
    const long long fs = op.ncls;
    const T* fg = op.fg + col.cls + (long long)k0 * fs;
    const T* fe = op.fe + col.cls + (long long)k0 * fs;
    const long long pl = op.plane;
    T yv[LZ], gv[LZ], ev[LZ];
    // all loads of the chunk first
    if (rsrc) {
        if (act) {
#pragma unroll
            for (int t = 0; t < LZ; ++t) {
                if (t < kn) {
                    yv[t] = fma(-alpha, qsrc[t * sstride], rsrc[t * sstride]);
                    gv[t] = ldro(fg + t * fs);
                    ev[t] = ldro(fe + t * fs);
                }
            }
        }
    } else if (full) {
#pragma unroll
        for (int t = 0; t < LZ; ++t) {
            yv[t] = fma(-alpha, qb[t * pl], rb[t * pl]);
            gv[t] = ldro(fg + t * fs);
            ev[t] = ldro(fe + t * fs);
        }
    } else if (act) {
#pragma unroll
        for (int t = 0; t < LZ; ++t) {
            if (t < kn) {
                yv[t] = fma(-alpha, qb[t * pl], rb[t * pl]);
                gv[t] = ldro(fg + t * fs);
                ev[t] = ldro(fe + t * fs);
            }
        }
    }
    const T e_in = (act && k0 > 0) ? ldro(fe - fs) * ldro(fg - fs) : T(0);
    // ZMODE 2 updates z in place: its old values are read with the chunk's
    // other loads (the thread owns them), not one by one after each store
    T zo[ZMODE == 2 ? LZ : 1];
    if constexpr (ZMODE == 2) {
        if (act) {
#pragma unroll
            for (int t = 0; t < LZ; ++t)
                if (t < kn) zo[t] = zb[t * pl];
        }
    }
    // updated residual, ||r||^2, local forward sweep with zero carry-in.
    // ||r||^2 and kappa are sums of non-negative terms: each chunk sums its
    // LZ terms directly (relative error <= (LZ - 1) u) and adds the chunk sum
    // to the compensated accumulator once.
    T yl = T(0), cp = T(0);
    if (act) {
        T ep = e_in;
        T rr_chunk = T(0);
#pragma unroll
        for (int t = 0; t < LZ; ++t) {
            if (t < kn) {
                const T rn = yv[t];
                if (STORE_R) rb[t * pl] = rn;
                rr_chunk = fma(rn, rn, rr_chunk);
                yl = fma(-ep, yl, rn) + yl;
                cp = (t == 0) ? ep : fma(ep, T(1) - cp, cp);
                yv[t] = yl;
                ep = ev[t] * gv[t];
            }
        }
        acc[0].add(rr_chunk);
    }
    sh_y[w0 + ch][lane] = yl;
    sh_c[w0 + ch][lane] = cp;
    __syncthreads();
    T Y = T(0);
    for (int cc = 0; cc < ch; ++cc) Y = fma(-sh_c[w0 + cc][lane], Y, sh_y[w0 + cc][lane]) + Y;
    // corrected y, kappa, then the local backward sweep with zero carry-in
    T zl = T(0), dp = T(0);
    if (act) {
        T ep = e_in;
        cp = T(0);
        T kap_chunk = T(0);
#pragma unroll
        for (int t = 0; t < LZ; ++t) {
            if (t < kn) {
                cp = (t == 0) ? ep : fma(ep, T(1) - cp, cp);
                const T y = fma(-cp, Y, yv[t]) + Y;
                yv[t] = y;
                kap_chunk = fma(gv[t] * y, y, kap_chunk);
                ep = ev[t] * gv[t];
            }
        }
        acc[1].add(kap_chunk);
        bool first = true;
#pragma unroll
        for (int t = LZ - 1; t >= 0; --t) {
            if (t < kn) {
                zl = fma(gv[t], fma(-ev[t], zl, yv[t]), zl);
                const T e = ev[t] * gv[t];
                dp = first ? e : fma(e, T(1) - dp, dp);
                first = false;
                yv[t] = zl;
            }
        }
    }
    sh_z[w0 + ch][lane] = zl;
    sh_d[w0 + ch][lane] = dp;
    __syncthreads();
    T Z = T(0);
    for (int cc = nch - 1; cc > ch; --cc) Z = fma(-sh_d[w0 + cc][lane], Z, sh_z[w0 + cc][lane]) + Z;
    if (act) {
        dp = T(0);
        bool first = true;
#pragma unroll
        for (int t = LZ - 1; t >= 0; --t) {
            if (t < kn) {
                const T e = ev[t] * gv[t];
                dp = first ? e : fma(e, T(1) - dp, dp);
                first = false;
                const T m = fma(-dp, Z, yv[t]) + Z;
                if constexpr (ZMODE == 0) zb[t * pl] = m;
                else if constexpr (ZMODE == 1) zb[t * pl] = omega * m;
                else zb[t * pl] = fma(omega, m, zo[t]);
            }
        }
    }
}

template <typename T, int LZ, int MINB = 1>
__global__ __launch_bounds__(256, MINB) void k_sweep_prec_chunked(OpView<T> op, T* __restrict__ r, const T* __restrict__ q,
                                                            T* __restrict__ z, SolveState* __restrict__ states,
                                                            double* __restrict__ partials,
                                                            unsigned* __restrict__ counters, int nblocks) {
    __shared__ T sh_y[MAXW][32], sh_c[MAXW][32], sh_z[MAXW][32], sh_d[MAXW][32];
    const int rhs = blockIdx.z;
    SolveState* st = states + rhs;
    if (st->done) return;
    const T alpha = (T)st->alpha;
    const int lane = threadIdx.x, ch = threadIdx.y, nch = blockDim.y;
    const Col<T> col = make_col(op, blockIdx.x * 32 + lane, blockIdx.y);
    const long long rb = (long long)rhs * op.vol;
    Acc<T> acc[2];
    prec_chunked_body<T, LZ>(op, col, lane, ch, nch, 0, r + rb, q + rb, z + rb, alpha, acc, sh_y, sh_c, sh_z, sh_d);
    double v[2];
    if (grid_sum_acc<2>(acc, partials + (long long)rhs * nblocks * 2, counters + rhs, nblocks, bid2(), v))
        prec_epilogue(st, v[0], v[1]);
}

// SpMV sweep: block = 32 x 4 columns, one chunk of LZ levels;
// blockIdx.z = rhs * nchunks + chunk.  The horizontal neighbours are read
// through the read-only cache; every load of a full chunk is issued before
// the arithmetic.
template <typename T, int LZ, int MINB = 1>
__global__ __launch_bounds__(NT, MINB) void k_sweep_spmv_chunked(OpView<T> op, T* __restrict__ u, T* __restrict__ p,
                                                           T* __restrict__ q, const T* __restrict__ z,
                                                           SolveState* __restrict__ states,
                                                           double* __restrict__ partials,
                                                           unsigned* __restrict__ counters, int nblocks, int nchunks) {
    const int rhs = blockIdx.z / nchunks;
    const int ch = blockIdx.z - rhs * nchunks;
    SolveState* st = states + rhs;
    if (st->done) return;
    const T alpha = (T)st->alpha;
    const T beta = (T)st->beta;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
    const Col<T> col = make_col(op, i0 + tx, j0 + ty);
    const int k0 = ch * LZ;
    const int kn = min(LZ, op.nz - k0);
    const long long pl = op.plane;
    const long long base = (long long)rhs * op.vol;
    const T* __restrict__ zb = z + base;
    T ur[LZ], pr[LZ], qr[LZ], zr[LZ + 2];
    const bool act = col.valid && kn > 0;
    T* ub = u + base + col.c + (long long)k0 * pl;
    T* pb = p + base + col.c + (long long)k0 * pl;
    T* qb = q + base + col.c + (long long)k0 * pl;
    if (act && kn == LZ) {
#pragma unroll
        for (int t = 0; t < LZ; ++t) {
            ur[t] = ub[t * pl];
            pr[t] = pb[t * pl];
            qr[t] = qb[t * pl];
            zr[t + 1] = ldro(zb + (long long)(k0 + t) * pl + col.c);
        }
        zr[0] = k0 > 0 ? ldro(zb + (long long)(k0 - 1) * pl + col.c) : T(0);
        zr[LZ + 1] = (k0 + LZ < op.nz) ? ldro(zb + (long long)(k0 + LZ) * pl + col.c) : zr[LZ];
    } else if (act) {
#pragma unroll
        for (int t = 0; t < LZ; ++t) {
            if (t < kn) {
                ur[t] = ub[t * pl];
                pr[t] = pb[t * pl];
                qr[t] = qb[t * pl];
                zr[t + 1] = ldro(zb + (long long)(k0 + t) * pl + col.c);
            }
        }
        zr[0] = k0 > 0 ? ldro(zb + (long long)(k0 - 1) * pl + col.c) : T(0);
    }
    Acc<T> sig[1];
    if (act) {
        T zc = zr[1];
        T fprev = (k0 > 0) ? ldro(op.wv + k0 - 1) * (zr[0] - zc) : T(0);
#pragma unroll
        for (int t = 0; t < LZ; ++t) {
            if (t < kn) {
                const int k = k0 + t;
                const T zu = (k + 1 < op.nz) ? (t + 1 < kn ? zr[t + 2] : zr[LZ + 1]) : zc;
                ub[t * pl] = fma(alpha, pr[t], ur[t]);
                const T pn = fma(beta, pr[t], zc);
                pb[t * pl] = pn;
                const T f = ldro(op.wv + k) * (zc - zu);
                const T hz = horiz(col, zb + (long long)k * pl, zc);
                const T az = fma(ldro(op.dk + k), hz, col.area * fma(ldro(op.mass + k), zc, f - fprev));
                const T qn = fma(beta, qr[t], az);
                qb[t * pl] = qn;
                sig[0].add_prod(pn, qn);
                fprev = f;
                zc = zu;
            }
        }
    }
    double v[1];
    const int bid = (ch * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (grid_sum_acc<1>(sig, partials + (long long)rhs * nblocks * 2, counters + rhs, nblocks, bid, v))
        spmv_epilogue(st, v[0]);
}


// ---------------------------------------------------------------------------
// FP32 SpMV sweep with TMA-staged tiles.
//
// Block = 32 x BYT columns, one chunk of LZ levels (blockIdx.z = rhs *
// nchunks + chunk).  One thread issues four bulk tensor copies into shared
// memory, all completing on one mbarrier:
//   z: levels k0-1 .. k0+LZ, columns i0-4 .. i0+35, rows j0-1 .. j0+BYT
//      (the stencil's one-cell halo; x starts 4 columns early so that the
//      copy starts on a 16-byte boundary),
//   u, p, q: levels k0 .. k0+LZ-1 of the block's own columns.
// Cells outside the grid arrive as zeros; a neighbour that wraps around a
// periodic edge (or is clamped at a Neumann edge) is read from global memory
// instead.  The right-hand side index is folded into the level coordinate,
// so the tensor maps describe [nrhs * n_z][n_y][n_x] arrays.  Arithmetic as
// in spmv_column<float>.
// ---------------------------------------------------------------------------
constexpr int TMA_HALO_X = 4;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void* tmap, int c0, int c1, int c2, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(c0), "r"(c1), "r"(c2), "r"(bar) : "memory");
}

// Wait for the phase with parity `parity` of the mbarrier at `bar`, giving up
// after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit) {
    for (int it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}
__device__ __forceinline__ bool mbar_wait0(uint32_t bar, int limit) { return mbar_wait(bar, 0u, limit); }

__device__ __forceinline__ void mbar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}

// Programmatic dependent launch: a sweep launched with programmatic stream
// serialization may start while the sweep before it drains.  Everything it
// does before pdl_wait() must not read what earlier sweeps wrote; pdl_wait()
// returns once the previous grid has completed and its writes are visible
// (at once when the launch had no such dependency).  pdl_trigger() lets the
// next sweep launch; it comes after pdl_wait(), so a sweep two launches back
// is always complete when a sweep starts.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <int LZ, int BYT>
struct SpmvTmaTile {
    static constexpr int ZX = BX + 2 * TMA_HALO_X, ZY = BYT + 2, ZZ = LZ + 2;
    static constexpr int ZN = ZX * ZY * ZZ, VN = BX * BYT * LZ;
    static constexpr uint32_t BYTES = (uint32_t)(ZN + 3 * VN) * 4u;
    static constexpr size_t SMEM = (size_t)BYTES + 16 + 128;   // + the mbarrier, + alignment slack
};

// The SpMV arithmetic of one thread on a staged tile (spmv_column<float>'s
// order of operations): zs holds levels k0-1 .. k0+LZ of the tile with halo,
// us/ps/qs levels k0 .. k0+LZ-1 of the block's own columns; z, u, p, q point
// at level 0 of the right-hand side.
template <int LZ, int BYT>
__device__ __forceinline__ void spmv_tile_compute(const OpView<float>& op, const Col<float>& col, int tx, int ty,
                                                  int k0, int kn, const float* zs, const float* us, const float* ps,
                                                  const float* qs, const float* __restrict__ z, float* __restrict__ u,
                                                  float* __restrict__ p, float* __restrict__ q, float alpha,
                                                  float beta, bool in_e, bool in_w, bool in_n, bool in_s,
                                                  Acc<float>& sig) {
    using TT = SpmvTmaTile<LZ, BYT>;
    const long long pl = op.plane;
    float* ub = u + col.c + (long long)k0 * pl;
    float* pb = p + col.c + (long long)k0 * pl;
    float* qb = q + col.c + (long long)k0 * pl;
    constexpr int ZX = TT::ZX, ZP = TT::ZX * TT::ZY;
    const int c0 = (ty + 1) * ZX + (tx + TMA_HALO_X);
    const int v0 = ty * BX + tx;
    float zc = zs[ZP + c0];
    float fprev = (k0 > 0) ? ldro(op.wv + k0 - 1) * (zs[c0] - zc) : 0.f;
#pragma unroll 4
    for (int t = 0; t < LZ; ++t) {
        if (t < kn) {
            const int k = k0 + t;
            const float* zl = zs + (t + 1) * ZP;
            const float zu = (k + 1 < op.nz) ? zl[ZP + c0] : zc;
            const float pk = ps[t * BX * BYT + v0];
            ub[t * pl] = fmaf(alpha, pk, us[t * BX * BYT + v0]);
            const float pn = fmaf(beta, pk, zc);
            pb[t * pl] = pn;
            const float f = ldro(op.wv + k) * (zc - zu);
            const float* zk = z + (long long)k * pl;
            const float ze = in_e ? zl[c0 + 1] : ldro(zk + col.ce);
            const float zw = in_w ? zl[c0 - 1] : ldro(zk + col.cw);
            const float zn = in_n ? zl[c0 + ZX] : ldro(zk + col.cn);
            const float zs_ = in_s ? zl[c0 - ZX] : ldro(zk + col.cs);
            float hz = col.me * (zc - ze);
            hz = fmaf(col.mw, zc - zw, hz);
            hz = fmaf(col.mn, zc - zn, hz);
            hz = fmaf(col.ms, zc - zs_, hz);
            const float az = fmaf(ldro(op.dk + k), hz, col.area * fmaf(ldro(op.mass + k), zc, f - fprev));
            const float qn = fmaf(beta, qs[t * BX * BYT + v0], az);
            qb[t * pl] = qn;
            sig.add_prod(pn, qn);
            fprev = f;
            zc = zu;
        }
    }
}

// Values a staged z tile lacks: neighbours across a periodic edge.  The
// bulk copy fills cells outside the grid with zeros, so a block on an edge
// loads the wrapped neighbours of its own cells (levels k0 .. k0+kn-1) from
// global memory into registers before its copies land, and writes them into
// the tile's halo (or, in a ragged last tile, into the cell just past the
// grid) once they have.  A face on a Neumann edge has weight 0, so its halo
// cell may keep the zero.  Thread (tx, ty) takes the x-wrap cells of level tx
// (< LZ) in row ty, and the y-wrap cells of column tx at levels ty, ty + BYT, ...
template <int LZ, int BYT>
struct WrapPatch {
    static constexpr int NY = (LZ + BYT - 1) / BYT;
    float xw, xe, ys[NY], yn[NY];
    bool any;            // block-uniform: the tile has a wrapped neighbour
    int i0, j0, nxv, nyv, kn;
    bool west, east, south, north;

    __device__ __forceinline__ void load(const OpView<float>& op, const float* __restrict__ zr, int i0_, int j0_,
                                         int k0, int kn_, int tx, int ty) {
        i0 = i0_;
        j0 = j0_;
        kn = kn_;
        nxv = min(BX, op.nx - i0);
        nyv = min(BYT, op.ny - j0);
        west = i0 == 0;
        east = i0 + BX >= op.nx;
        south = op.periodic_y && j0 == 0;
        north = op.periodic_y && j0 + BYT >= op.ny;
        any = west || east || south || north;
        if (!any) return;
        const long long pl = op.plane, nx = op.nx;
        if (tx < kn && ty < nyv) {
            const float* lev = zr + (long long)(k0 + tx) * pl + (long long)(j0 + ty) * nx;
            if (west) xw = ldro(lev + (nx - 1));
            if (east) xe = ldro(lev);
        }
        if (tx < nxv) {
#pragma unroll
            for (int m = 0; m < NY; ++m) {
                const int t = ty + m * BYT;
                if (t < kn) {
                    const float* lev = zr + (long long)(k0 + t) * pl + (i0 + tx);
                    if (south) ys[m] = ldro(lev + (long long)(op.ny - 1) * nx);
                    if (north) yn[m] = ldro(lev);
                }
            }
        }
    }

    // zs: the tile [LZ+2][BYT+2][BX+2*TMA_HALO_X], level t of the chunk at t+1
    __device__ __forceinline__ void store(float* zs, int tx, int ty) const {
        constexpr int ZX = BX + 2 * TMA_HALO_X, ZP = ZX * (BYT + 2);
        if (tx < kn && ty < nyv) {
            float* row = zs + (tx + 1) * ZP + (ty + 1) * ZX + TMA_HALO_X;
            if (west) row[-1] = xw;
            if (east) row[nxv] = xe;
        }
        if (tx < nxv) {
#pragma unroll
            for (int m = 0; m < NY; ++m) {
                const int t = ty + m * BYT;
                if (t < kn) {
                    float* lev = zs + (t + 1) * ZP + TMA_HALO_X + tx;
                    if (south) lev[0] = ys[m];
                    if (north) lev[(nyv + 1) * ZX] = yn[m];
                }
            }
        }
    }
};

// The SpMV arithmetic of one thread on a staged tile whose halo holds every
// neighbour (WrapPatch applied), in spmv_column<float>'s order of operations:
// zs holds levels k0-1 .. k0+LZ of the tile with halo, us/ps/qs levels k0 ..
// k0+LZ-1 of the block's own columns; tw[t], td[t], tm[t] are wv, dk and mass
// at level k0 + t (tw[-1] too when k0 > 0); u, p, q point at level 0 of the
// right-hand side.  With S > 1 the chunk's levels are split among S threads
// of the same column: this one takes levels part LZ/S .. (part + 1) LZ/S - 1
// and forms the flux below its first level from the tile itself (the same
// operands and operations as the thread below it, so every cell's result is
// the same for any S).  sigma = <p, q> of the thread's levels is summed in
// plain FP32 (error <= (LZ/S) u sum_k |p_k q_k|) and added to the compensated
// accumulator once.
template <int LZ, int BYT, int S = 1>
__device__ __forceinline__ void spmv_tile_compute_p(const OpView<float>& op, const Col<float>& col, int tx, int ty,
                                                    int k0, int kn, const float* zs, const float* us,
                                                    const float* ps, const float* qs, const float* tw,
                                                    const float* td, const float* tm, float* __restrict__ u,
                                                    float* __restrict__ p, float* __restrict__ q, float alpha,
                                                    float beta, Acc<float>& sig, int part = 0) {
    using TT = SpmvTmaTile<LZ, BYT>;
    constexpr int LH = LZ / S;                  // levels of this thread: part LH .. part LH + LH - 1 of the chunk
    const int t0 = part * LH;
    if (t0 >= kn) return;
    const long long pl = op.plane;
    float* __restrict__ ub = u + col.c + (long long)k0 * pl;
    float* __restrict__ pb = p + col.c + (long long)k0 * pl;
    float* __restrict__ qb = q + col.c + (long long)k0 * pl;
    constexpr int ZX = TT::ZX, ZP = TT::ZX * TT::ZY;
    const int c0 = (ty + 1) * ZX + (tx + TMA_HALO_X);
    const int v0 = ty * BX + tx;
    const bool top = k0 + kn == op.nz;          // the chunk holds the top level: no flux above it
    float zc = zs[(t0 + 1) * ZP + c0];
    float fprev = (k0 + t0 > 0) ? tw[t0 - 1] * (zs[t0 * ZP + c0] - zc) : 0.f;
    float sc = 0.f;
#pragma unroll
    for (int tt = 0; tt < LH; ++tt) {
        const int t = t0 + tt;
        if (t < kn) {
            const float* zl = zs + (t + 1) * ZP;
            const float zu = (top && t + 1 == kn) ? zc : zl[ZP + c0];
            const float pk = ps[t * BX * BYT + v0];
            ub[t * pl] = fmaf(alpha, pk, us[t * BX * BYT + v0]);
            const float pn = fmaf(beta, pk, zc);
            pb[t * pl] = pn;
            const float f = tw[t] * (zc - zu);
            float hz = col.me * (zc - zl[c0 + 1]);
            hz = fmaf(col.mw, zc - zl[c0 - 1], hz);
            hz = fmaf(col.mn, zc - zl[c0 + ZX], hz);
            hz = fmaf(col.ms, zc - zl[c0 - ZX], hz);
            const float az = fmaf(td[t], hz, col.area * fmaf(tm[t], zc, f - fprev));
            const float qn = fmaf(beta, qs[t * BX * BYT + v0], az);
            qb[t * pl] = qn;
            sc = fmaf(pn, qn, sc);
            fprev = f;
            zc = zu;
        }
    }
    sig.add(sc);
}

template <int LZ, int BYT>
__global__ __launch_bounds__(BX * BYT) void k_sweep_spmv_tma(
    OpView<float> op, const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_p,
    const __grid_constant__ CUtensorMap tm_q, const __grid_constant__ CUtensorMap tm_z, float* __restrict__ u,
    float* __restrict__ p, float* __restrict__ q, const float* __restrict__ z, SolveState* __restrict__ states,
    double* __restrict__ partials, unsigned* __restrict__ counters, int nblocks, int nchunks) {
    using TT = SpmvTmaTile<LZ, BYT>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ float tb[3][LZ + 1];         // wv at k0-1 .. k0+LZ-1, dk and mass at k0 .. k0+LZ-1
    // bulk tensor copies land on 128-byte aligned addresses
    float* zs = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));   // [ZZ][ZY][ZX]
    float* us = zs + TT::ZN;                // [LZ][BYT][32]
    float* ps = us + TT::VN;
    float* qs = ps + TT::VN;
    uint64_t* bar = reinterpret_cast<uint64_t*>(qs + TT::VN);
    const int rhs = blockIdx.z / nchunks;
    const int ch = blockIdx.z - rhs * nchunks;
    SolveState* st = states + rhs;
    if (st->done) return;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BYT;
    const int k0 = ch * LZ;
    const int kn = min(LZ, op.nz - k0);
    const int lev0 = rhs * op.nz + k0;      // level coordinate of the chunk in the folded arrays
    const uint32_t b = smem_u32(bar);
    if (tid == 0) mbar_init(b);
    __syncthreads();
    if (tid == 0) {
        mbar_expect(b, TT::BYTES);
        tma_load_3d(smem_u32(zs), &tm_z, i0 - TMA_HALO_X, j0 - 1, lev0 - 1, b);
        tma_load_3d(smem_u32(us), &tm_u, i0, j0, lev0, b);
        tma_load_3d(smem_u32(ps), &tm_p, i0, j0, lev0, b);
        tma_load_3d(smem_u32(qs), &tm_q, i0, j0, lev0, b);
    }
    // while the copies are in flight: level tables, column geometry, wrapped neighbours
    if (tid < 3 * (LZ + 1)) {
        const int a = tid / (LZ + 1), t = tid - a * (LZ + 1);
        const int k = k0 - 1 + t;
        const float* src = a == 0 ? op.wv : (a == 1 ? op.dk : op.mass);
        const int ko = a == 0 ? k : k + 1;  // dk, mass: entry t is level k0 + t
        tb[a][t] = (ko >= 0 && ko < op.nz) ? ldro(src + ko) : 0.f;
    }
    const float alpha = (float)st->alpha;
    const float beta = (float)st->beta;
    const Col<float> col = make_col(op, i0 + tx, j0 + ty);
    const bool act = col.valid && kn > 0;
    const long long base = (long long)rhs * op.vol;
    WrapPatch<LZ, BYT> wp;
    wp.load(op, z + base, i0, j0, k0, kn, tx, ty);
    const bool landed = mbar_wait0(b, 1 << 22);
    if (landed) wp.store(zs, tx, ty);
    __syncthreads();
    Acc<float> sig[1];
    if (!landed) {
        // the copies did not complete in time: record it (the last block ends
        // the solve), wait (bounded) for them to land before the block's
        // shared memory is released, and add nothing to sigma
        if (tid == 0) atomicExch(&st->status, 6);   // PCG_TIMEOUT
        mbar_wait0(b, 1 << 22);
    } else if (act) {
        spmv_tile_compute_p<LZ, BYT>(op, col, tx, ty, k0, kn, zs, us, ps, qs, &tb[0][1], tb[1], tb[2], u + base,
                                     p + base, q + base, alpha, beta, sig[0]);
    }
    double v[1];
    const int bid = (ch * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (grid_sum_acc<1>(sig, partials + (long long)rhs * nblocks * 2, counters + rhs, nblocks, bid, v))
        spmv_epilogue(st, v[0]);
}

// ---------------------------------------------------------------------------
// The same SpMV sweep as a persistent two-stage pipeline: blockIdx.y = right-
// hand side; a block walks the (tile, chunk) items i = blockIdx.x, +gridDim.x,
// ... and keeps the copies of its next item in flight (second stage, second
// mbarrier) while it computes the current one.  The level tables of all n_z
// levels sit in shared memory after the two stages; the grid-level reduction
// runs once per block instead of once per item.  Blocks are BX x (BYT S)
// threads: S threads per column, each taking LZ/S levels of the chunk, so a
// block has S times the warps to hide the latency of its shared-memory reads
// and of the dependent chain of each column (S = 2 at 256^2 x 128: 54.3 ->
// 51.0 us per sweep; 1024^2 x 128: 650 -> 621 us).
// ---------------------------------------------------------------------------
template <int LZ, int BYT>
__host__ __device__ constexpr size_t spmv_tma2_smem(int nz) {
    return 2 * ((size_t)SpmvTmaTile<LZ, BYT>::ZN + 3 * SpmvTmaTile<LZ, BYT>::VN) * 4 + (size_t)(3 * nz + 4) * 4 + 16 +
           128;
}

template <int LZ, int BYT, int S = 1>
__global__ __launch_bounds__(BX * BYT * S) void k_sweep_spmv_tma2(
    OpView<float> op, const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_p,
    const __grid_constant__ CUtensorMap tm_q, const __grid_constant__ CUtensorMap tm_z, float* __restrict__ u,
    float* __restrict__ p, float* __restrict__ q, const float* __restrict__ z, SolveState* __restrict__ states,
    double* __restrict__ partials, unsigned* __restrict__ counters, int gx, int gy, int nchunks) {
    using TT = SpmvTmaTile<LZ, BYT>;
    constexpr int STAGE = TT::ZN + 3 * TT::VN;          // floats per stage (a multiple of 32)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* sbase = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int nz = op.nz;
    float* tbw = sbase + 2 * STAGE;                     // wv[0 .. nz-1] at tbw[1 ..], tbw[0] = 0
    float* tbd = tbw + nz + 1;
    float* tbm = tbd + nz;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sbase + 2 * STAGE + ((3 * nz + 4) & ~3));
    const int rhs = blockIdx.y;
    SolveState* st = states + rhs;
    // block (BX, BYT * S): row ty of the tile, level part tz of the chunk
    const int tx = threadIdx.x, ty = threadIdx.y % BYT, tz = threadIdx.y / BYT, tid = threadIdx.y * BX + tx;
    const int nitems = gx * gy * nchunks;
    const uint32_t bar0 = smem_u32(bars), bar1 = smem_u32(bars + 1);
    // prologue on data no sweep writes (it may overlap the previous sweep)
    if (tid == 0) {
        mbar_init(bar0);
        mbar_init(bar1);
    }
    for (int k = tid; k < nz; k += BX * BYT * S) {
        tbw[k + 1] = ldro(op.wv + k);
        tbd[k] = ldro(op.dk + k);
        tbm[k] = ldro(op.mass + k);
    }
    if (tid == 0) tbw[0] = 0.f;
    __syncthreads();
    pdl_wait();
    pdl_trigger();
    if (st->done) return;
    auto issue = [&](int item, int stage) {
        const int ch = item % nchunks, tile = item / nchunks;
        const int i0 = (tile % gx) * BX, j0 = (tile / gx) * BYT, lev0 = rhs * nz + ch * LZ;
        float* zs = sbase + stage * STAGE;
        const uint32_t bar = stage ? bar1 : bar0;
        mbar_expect(bar, TT::BYTES);
        tma_load_3d(smem_u32(zs), &tm_z, i0 - TMA_HALO_X, j0 - 1, lev0 - 1, bar);
        tma_load_3d(smem_u32(zs + TT::ZN), &tm_u, i0, j0, lev0, bar);
        tma_load_3d(smem_u32(zs + TT::ZN + TT::VN), &tm_p, i0, j0, lev0, bar);
        tma_load_3d(smem_u32(zs + TT::ZN + 2 * TT::VN), &tm_q, i0, j0, lev0, bar);
    };
    uint32_t pending = 0;
    if ((int)blockIdx.x < nitems) {
        if (tid == 0) issue(blockIdx.x, 0);
        pending |= 1u;
    }
    if ((int)(blockIdx.x + gridDim.x) < nitems) {
        if (tid == 0) issue(blockIdx.x + gridDim.x, 1);
        pending |= 2u;
    }
    const float alpha = (float)st->alpha;
    const float beta = (float)st->beta;
    const long long base = (long long)rhs * op.vol;
    Acc<float> sig[1];
    uint32_t par0 = 0, par1 = 0;
    bool ok = true;                 // false once a stage failed to land in time
    int n = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++n) {
        const int stage = n & 1;
        const int ch = item % nchunks, tile = item / nchunks;
        const int i0 = (tile % gx) * BX, j0 = (tile / gx) * BYT, k0 = ch * LZ;
        const int kn = min(LZ, nz - k0);
        WrapPatch<LZ, BYT> wp;
        wp.load(op, z + base, i0, j0, k0, tz == 0 ? kn : 0, tx, ty);   // the first level part patches the halo
        const Col<float> col = make_col(op, i0 + tx, j0 + ty);
        bool landed = mbar_wait(stage ? bar1 : bar0, stage ? par1 : par0, 1 << 22);
        landed = __syncthreads_and(landed ? 1 : 0) != 0;
        if (!landed) {
            if (tid == 0) atomicExch(&st->status, 6);   // PCG_TIMEOUT
            ok = false;
            break;
        }
        if (stage) par1 ^= 1u; else par0 ^= 1u;
        pending &= ~(1u << stage);
        float* zs = sbase + stage * STAGE;
        if (wp.any) {
            wp.store(zs, tx, ty);
            __syncthreads();
        }
        if (col.valid && kn > 0)
            spmv_tile_compute_p<LZ, BYT, S>(op, col, tx, ty, k0, kn, zs, zs + TT::ZN, zs + TT::ZN + TT::VN,
                                            zs + TT::ZN + 2 * TT::VN, tbw + 1 + k0, tbd + k0, tbm + k0, u + base,
                                            p + base, q + base, alpha, beta, sig[0], tz);
        // the stage has been read (and patched) by the threads: order that
        // before the bulk copies that refill it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (item + 2 * (int)gridDim.x < nitems) {
            if (tid == 0) issue(item + 2 * gridDim.x, stage);
            pending |= 1u << stage;
        }
    }
    if (!ok) {
        if (pending & 1u) mbar_wait(bar0, par0, 1 << 22);
        if (pending & 2u) mbar_wait(bar1, par1, 1 << 22);
    }
    double v[1];
    if (grid_sum_acc<1>(sig, partials + (long long)rhs * gridDim.x * 2, counters + rhs, gridDim.x, blockIdx.x, v))
        spmv_epilogue(st, v[0]);
}

// ---------------------------------------------------------------------------
// FP32 preconditioner sweep on a TMA pipeline: the chunked solve of
// prec_chunked_body on tiles staged in shared memory.
//
// Persistent blocks of 256 threads, blockIdx.y = right-hand side.  An item
// is R rows of 32 columns over all levels (R * nch <= 8: warp w takes row
// w / nch, chunk w % nch).  One thread streams the items' r and q tiles
// ([LEV][R][32], LEV = nch * LZ) into two shared-memory stages by bulk
// tensor copies, each stage on its own mbarrier, so the copies of the next
// item are in flight while an item is solved.  The threads write r and z.
// ---------------------------------------------------------------------------
template <int LZ>
struct PrecTmaTile {
    static constexpr int VN = 8 * LZ * 32;                 // floats of one vector in one stage (R * LEV <= 8 LZ)
    static constexpr size_t SMEM = 4 * (size_t)VN * 4 + 16 + 128;   // 2 stages x (r, q), 2 mbarriers, alignment
};

// Per-level tables of the chunked preconditioner when every column has the
// same factors (cls_mode 0, n_z <= 8 LZ): 1/D, E, e = E/D and the carry
// weights of each level's LZ-level chunk, C (forward: 1 - prod of (1 - e)
// from the chunk's first level up) and Q (backward: from the chunk's last
// level down).  Each block builds them from the FP32 factors with exactly
// the operations prec_chunked_body repeats per column and pass, so the solve
// is bitwise that of prec_chunked_body at a fraction of the instructions.
template <int LZ>
struct PrecTab {
    float g[8 * LZ], E[8 * LZ], e[8 * LZ], C[8 * LZ], Q[8 * LZ];
};

template <int LZ>
__device__ __forceinline__ void prec_tab_build(const OpView<float>& op, PrecTab<LZ>& tb, int tid, int nthr) {
    const int nz = op.nz;
    for (int k = tid; k < nz; k += nthr) {
        const float g = ldro(op.fg + k), E = ldro(op.fe + k);   // one factor set: ncls == 1
        tb.g[k] = g;
        tb.E[k] = E;
        tb.e[k] = E * g;
    }
    __syncthreads();
    const int nch = (nz + LZ - 1) / LZ;
    if (tid < nch) {
        const int k0 = tid * LZ, kn = min(LZ, nz - k0);
        float cp = k0 > 0 ? tb.e[k0 - 1] : 0.f;
        tb.C[k0] = cp;
        for (int t = 1; t < kn; ++t) {
            cp = fmaf(tb.e[k0 + t - 1], 1.f - cp, cp);
            tb.C[k0 + t] = cp;
        }
        float dp = tb.e[k0 + kn - 1];
        tb.Q[k0 + kn - 1] = dp;
        for (int t = kn - 2; t >= 0; --t) {
            dp = fmaf(tb.e[k0 + t], 1.f - dp, dp);
            tb.Q[k0 + t] = dp;
        }
    }
    __syncthreads();
}

// prec_chunked_body on a staged tile with the tables above: the chunk's r and
// q at rsrc[t R 32], qsrc[t R 32]; FULL: the chunk has LZ levels.  Holds two
// block barriers, like prec_chunked_body.
template <int LZ, int R, bool FULL>
__device__ __forceinline__ void prec_tab_body(const OpView<float>& op, const PrecTab<LZ>& tb, const Col<float>& col,
                                              int lane, int ch, int nch, int w0, float* __restrict__ r,
                                              float* __restrict__ z, float alpha, Acc<float> (&acc)[2],
                                              float (*sh_y)[32], float (*sh_c)[32], float (*sh_z)[32],
                                              float (*sh_d)[32], const float* rsrc, const float* qsrc) {
    const int k0 = ch * LZ;
    const int kn = FULL ? LZ : min(LZ, op.nz - k0);
    const bool act = col.valid && kn > 0;
    const long long pl = op.plane;
    float* __restrict__ rb = r + col.c + (long long)k0 * pl;
    float* __restrict__ zb = z + col.c + (long long)k0 * pl;
    float yv[LZ];
    float yl = 0.f;
    if (act) {
        const float e_in = k0 > 0 ? tb.e[k0 - 1] : 0.f;
        float rr_c = 0.f;
#pragma unroll
        for (int t = 0; t < LZ; ++t) {
            if (FULL || t < kn) {
                const float rn = fmaf(-alpha, qsrc[t * R * 32], rsrc[t * R * 32]);
                rb[t * pl] = rn;
                rr_c = fmaf(rn, rn, rr_c);
                const float ep = t == 0 ? e_in : tb.e[k0 + t - 1];
                yl = fmaf(-ep, yl, rn) + yl;
                yv[t] = yl;
            }
        }
        acc[0].add(rr_c);
    }
    sh_y[w0 + ch][lane] = yl;
    sh_c[w0 + ch][lane] = act ? tb.C[k0 + kn - 1] : 0.f;
    __syncthreads();
    float Y = 0.f;
    for (int cc = 0; cc < ch; ++cc) Y = fmaf(-sh_c[w0 + cc][lane], Y, sh_y[w0 + cc][lane]) + Y;
    float zl = 0.f;
    if (act) {
        float kap_c = 0.f;
#pragma unroll
        for (int t = 0; t < LZ; ++t) {
            if (FULL || t < kn) {
                const float y = fmaf(-tb.C[k0 + t], Y, yv[t]) + Y;
                yv[t] = y;
                kap_c = fmaf(tb.g[k0 + t] * y, y, kap_c);
            }
        }
        acc[1].add(kap_c);
#pragma unroll
        for (int t = LZ - 1; t >= 0; --t) {
            if (FULL || t < kn) {
                zl = fmaf(tb.g[k0 + t], fmaf(-tb.E[k0 + t], zl, yv[t]), zl);
                yv[t] = zl;
            }
        }
    }
    sh_z[w0 + ch][lane] = zl;
    sh_d[w0 + ch][lane] = act ? tb.Q[k0] : 0.f;
    __syncthreads();
    float Z = 0.f;
    for (int cc = nch - 1; cc > ch; --cc) Z = fmaf(-sh_d[w0 + cc][lane], Z, sh_z[w0 + cc][lane]) + Z;
    if (act) {
#pragma unroll
        for (int t = LZ - 1; t >= 0; --t)
            if (FULL || t < kn) zb[t * pl] = fmaf(-tb.Q[k0 + t], Z, yv[t]) + Z;
    }
}

// RT > 0: one factor set for all columns, tables (PrecTab) and items of RT rows
// known at compile time; RT == 0: any factor classes, prec_chunked_body.
template <int LZ, int RT>
__global__ __launch_bounds__(256, 2) void k_sweep_prec_tma(
    OpView<float> op, const __grid_constant__ CUtensorMap tm_r, const __grid_constant__ CUtensorMap tm_q,
    float* __restrict__ r, const float* __restrict__ q, float* __restrict__ z, SolveState* __restrict__ states,
    double* __restrict__ partials, unsigned* __restrict__ counters, int R, int nch, int gx, int nitems) {
    using TT = PrecTmaTile<LZ>;
    __shared__ float sh_y[MAXW][32], sh_c[MAXW][32], sh_z[MAXW][32], sh_d[MAXW][32];
    __shared__ PrecTab<(RT > 0 ? LZ : 1)> tb[1];
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* sbase = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint64_t* bars = reinterpret_cast<uint64_t*>(sbase + 4 * TT::VN);
    const int rhs = blockIdx.y;
    SolveState* st = states + rhs;
    if (RT > 0) R = RT;
    const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane;
    const int row = w / nch, ch = w - row * nch;
    const uint32_t bytes = 2u * 32u * (uint32_t)R * (uint32_t)(nch * LZ) * 4u;
    const uint32_t bar0 = smem_u32(bars), bar1 = smem_u32(bars + 1);
    // prologue on data no sweep writes (it may overlap the previous sweep):
    // the barriers and, with one factor set, the carry tables
    if (tid == 0) {
        mbar_init(bar0);
        mbar_init(bar1);
    }
    __syncthreads();
    if constexpr (RT > 0) prec_tab_build<LZ>(op, tb[0], tid, 256);
    pdl_wait();
    pdl_trigger();
    if (st->done) return;
    const float alpha = (float)st->alpha;
    const int lev0 = rhs * op.nz;
    auto issue = [&](int item, int stage) {
        const uint32_t bar = stage ? bar1 : bar0;
        float* rs = sbase + stage * 2 * TT::VN;
        mbar_expect(bar, bytes);
        tma_load_3d(smem_u32(rs), &tm_r, (item % gx) * 32, (item / gx) * R, lev0, bar);
        tma_load_3d(smem_u32(rs + TT::VN), &tm_q, (item % gx) * 32, (item / gx) * R, lev0, bar);
    };
    if (tid == 0) {
        if ((int)blockIdx.x < nitems) issue(blockIdx.x, 0);
        if ((int)(blockIdx.x + gridDim.x) < nitems) issue(blockIdx.x + gridDim.x, 1);
    }
    const long long vb = (long long)rhs * op.vol;
    Acc<float> acc[2];
    uint32_t par0 = 0, par1 = 0;
    bool ok = true;                 // false once a stage failed to land in time: nothing more is computed
    int n = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++n) {
        const int stage = n & 1;
        bool landed = false;
        if (ok) landed = mbar_wait(stage ? bar1 : bar0, stage ? par1 : par0, 1 << 22);
        landed = __syncthreads_and(landed ? 1 : 0) != 0;
        if (landed) {
            if (stage) par1 ^= 1u; else par0 ^= 1u;
        }
        if (ok && !landed) {
            if (tid == 0) atomicExch(&st->status, 6);   // PCG_TIMEOUT
            ok = false;
        }
        const int j = (ok && row < R) ? (item / gx) * R + row : op.ny;   // op.ny: no column (barriers only)
        const Col<float> col = make_col(op, (item % gx) * 32 + lane, j);
        const float* rs = sbase + stage * 2 * TT::VN + ((ch * LZ) * R + row) * 32 + lane;
        if constexpr (RT > 0) {
            if (ch * LZ + LZ <= op.nz)
                prec_tab_body<LZ, RT, true>(op, tb[0], col, lane, ch, nch, row * nch, r + vb, z + vb, alpha, acc,
                                            sh_y, sh_c, sh_z, sh_d, rs, rs + TT::VN);
            else
                prec_tab_body<LZ, RT, false>(op, tb[0], col, lane, ch, nch, row * nch, r + vb, z + vb, alpha, acc,
                                             sh_y, sh_c, sh_z, sh_d, rs, rs + TT::VN);
        } else {
            prec_chunked_body<float, LZ>(op, col, lane, ch, nch, row * nch, r + vb, q + vb, z + vb, alpha, acc, sh_y,
                                         sh_c, sh_z, sh_d, rs, rs + TT::VN, R * 32);
        }
        __syncthreads();            // the stage has been read: refill it
        if (tid == 0 && ok && item + 2 * (int)gridDim.x < nitems) issue(item + 2 * gridDim.x, stage);
    }
    if (!ok) {
        // copies still in flight (the pending phase of each stage) land before
        // the block's shared memory is released
        mbar_wait(bar0, par0, 1 << 22);
        mbar_wait(bar1, par1, 1 << 22);
    }
    double v[2];
    if (grid_sum_acc<2>(acc, partials + (long long)rhs * gridDim.x * 2, counters + rhs, gridDim.x, blockIdx.x, v))
        prec_epilogue(st, v[0], v[1]);
}

// ---------------------------------------------------------------------------
// Residual r = b - A x in FP64, with reductions of <b,b>, <r,r>, sum(r) and
// the rounding floor sum_i ulp(x_i)^2/12 ||A e_i||^2 (the expected squared
// residual of x rounded to FP64: no FP64 vector gets closer to b than this).
// mode 0: start of an FP64 solve: also u = x, writes r; sets the stopping threshold.
// mode 1: true residual after a solve: writes nothing, stores rr_true and floor2.
// mode 2: refinement, measure: writes nothing, stores bnorm2, rr, rsum, floor2.
// mode 3: refinement, emit: writes r' = b - A x - coarse * m (the inner
//         right-hand side, in TO) and stores <r', r'> in rr_emit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double ulp64(double x) {
    const long long e = (__double_as_longlong(x) >> 52) & 0x7ff;
    return e > 52 ? __longlong_as_double((e - 52) << 52) : 0.0;
}

template <typename TO>
__global__ __launch_bounds__(NT) void k_residual(OpView<double> op, const double* __restrict__ b,
                                                 const double* __restrict__ x, double* __restrict__ u,
                                                 TO* __restrict__ rout, SolveState* __restrict__ states,
                                                 double* __restrict__ partials, unsigned* __restrict__ counters,
                                                 int nblocks, int mode) {
    const int rhs = blockIdx.z;
    SolveState* st = states + rhs;
    const Col<double> col = make_col(op, blockIdx.x * BX + threadIdx.x, blockIdx.y * BY + threadIdx.y);
    const double coarse = (mode == 3) ? st->coarse : 0.0;
    const bool want_floor = (mode == 1 || mode == 2);
    double bb = 0.0, rr = 0.0, rs = 0.0, fl = 0.0;
    if (col.valid) {
        const long long base = (long long)rhs * op.vol;
        const double* __restrict__ xb = x + base;
        const double* __restrict__ bbp = b + base + col.c;
        const double hsum2 = col.me * col.me + col.mw * col.mw + col.mn * col.mn + col.ms * col.ms;
        const double hsum = (col.me + col.mw) + (col.mn + col.ms);
        double zc = xb[col.c];
        double fprev = 0.0, wprev = 0.0;
#pragma unroll 4
        for (int k = 0; k < op.nz; ++k) {
            const long long o = (long long)k * op.plane;
            const double* xl = xb + o;
            const double zu = (k + 1 < op.nz) ? ldro(xl + op.plane + col.c) : zc;
            const double wk = ldro(op.wv + k);
            const double f = wk * (zc - zu);
            const double hz = horiz(col, xl, zc);
            const double dk = ldro(op.dk + k);
            const double cm = col.area * ldro(op.mass + k);
            const double az = fma(dk, hz, col.area * fma(ldro(op.mass + k), zc, f - fprev));
            const double bv = bbp[o];
            const double rv = fma(-coarse, cm, bv - az);
            bb = fma(bv, bv, bb);
            rr = fma(rv, rv, rr);
            rs += rv;
            if (want_floor) {
                const double wu = col.area * wk, wd = col.area * wprev;
                const double diag = cm + dk * hsum + wu + wd;
                const double cn2 = diag * diag + dk * dk * hsum2 + wu * wu + wd * wd;
                const double ul = ulp64(zc);
                fl = fma(ul * ul, cn2, fl);
            }
            if (mode == 0) u[base + o + col.c] = zc;
            if (mode == 0 || mode == 3) rout[base + o + col.c] = (TO)rv;
            fprev = f;
            wprev = wk;
            zc = zu;
        }
    }
    double v[4] = {bb, rr, rs, fl / 12.0};
    if (grid_sum<4>(v, partials + (long long)rhs * nblocks * 4, counters + rhs, nblocks, bid2())) {
        if (mode == 0) {
            st->bnorm2 = v[0];
            st->rr = v[1];
            st->thresh2 = st->tol2 * v[0];
            if (v[0] == 0.0) {
                st->zero_rhs = 1;
                st->done = 1;
                st->status = 0;
            }
        } else if (mode == 1) {
            st->rr_true = v[1];
            st->floor2 = v[3];
        } else if (mode == 2) {
            st->bnorm2 = v[0];
            st->rr = v[1];
            st->rsum = v[2];
            st->floor2 = v[3];
        } else {
            st->rr_emit = v[1];
        }
    }
}

// Initialise the scalar state of nrhs solves.
__global__ void k_init_state(SolveState* states, int nrhs, double tol2, int maxit, const int* active) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    SolveState s;
    s.alpha = 0.0;
    s.beta = 0.0;
    s.kappa_old = 1.0;
    s.sigma = 0.0;
    s.rr = 0.0;
    s.kappa = 0.0;
    s.bnorm2 = 0.0;
    s.thresh2 = 0.0;
    s.tol2 = tol2;
    s.rr_true = 0.0;
    s.done = active ? (active[r] ? 0 : 1) : 0;
    s.status = 0;
    s.pass = 0;
    s.maxit = maxit;
    s.zero_rhs = 0;
    s.rsum = 0.0;
    s.coarse = 0.0;
    s.rr_emit = 0.0;
    s.floor2 = 0.0;
    s.pad_ = 0;
    states[r] = s;
}

// Inner-solve thresholds from the refinement residual: thresh2 = tol_in^2 <r', r'>.
__global__ void k_inner_thresholds(SolveState* inner, const SolveState* outer, int nrhs, double tol_in2) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    inner[r].thresh2 = tol_in2 * outer[r].rr_emit;
    inner[r].bnorm2 = outer[r].rr_emit;
}

// Coarse correction of one refinement sweep: the Galerkin projection of the
// residual onto the constant vector, c = sum(r) / sum(A 1) (A 1 is the mass
// vector exactly), so that the inner solve sees a residual orthogonal to 1.
__global__ void k_coarse(SolveState* states, int nrhs, double total_mass) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    states[r].coarse = total_mass > 0.0 ? states[r].rsum / total_mass : 0.0;
}

// Final update of an FP64 solve: x = u + alpha p (x = 0 for a zero right-hand side).
__global__ __launch_bounds__(NT) void k_finish(int nx, int ny, int nz, long long plane, long long vol,
                                               double* __restrict__ x, const double* __restrict__ u,
                                               const double* __restrict__ p, const SolveState* __restrict__ states) {
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i >= nx || j >= ny) return;
    const SolveState* st = states + blockIdx.z;
    const double alpha = st->alpha;
    const bool zero = st->zero_rhs != 0;
    const long long base = (long long)blockIdx.z * vol + (long long)j * nx + i;
    for (int k = 0; k < nz; ++k) {
        const long long o = base + (long long)k * plane;
        x[o] = zero ? 0.0 : fma(alpha, p[o], u[o]);
    }
}

// Refinement update x += coarse + u + alpha p (the coarse correction, the
// inner FP32 iterate and the deferred last step of Algorithm 1), for
// right-hand sides whose inner solve ran.
__global__ __launch_bounds__(NT) void k_refine_update(int nx, int ny, int nz, long long plane, long long vol,
                                                      double* __restrict__ x, const float* __restrict__ u,
                                                      const float* __restrict__ p, const SolveState* __restrict__ inner,
                                                      const SolveState* __restrict__ outer, const int* __restrict__ active) {
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i >= nx || j >= ny) return;
    if (!active[blockIdx.z]) return;
    const double alpha = inner[blockIdx.z].alpha;
    const double coarse = outer[blockIdx.z].coarse;
    const long long base = (long long)blockIdx.z * vol + (long long)j * nx + i;
    for (int k = 0; k < nz; ++k) {
        const long long o = base + (long long)k * plane;
        x[o] = fma(alpha, (double)p[o], (x[o] + coarse) + (double)u[o]);
    }
}

// Thomas factors of M for every factor class, in FP64, carrying the pivot as
// W_k + E_k with the excess E_k = s_k + W_{k-1} E_{k-1} / D_{k-1} >= 0
// (s_k: zero-order plus horizontal-diagonal part of row k).  No term is
// subtracted, so the pivots keep full relative accuracy however small s_k is
// next to the vertical couplings.  Stored per level and class: 1/D_k, E_k
// and, when fc is given, c_k = W_k / D_k for the FP64 sweeps.
__global__ void k_factors(OpView<double> op, double* __restrict__ fg, double* __restrict__ fe,
                          double* __restrict__ fc) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= op.ncls) return;
    int i = 0, j = 0;
    if (op.cls_mode == 1) j = c;
    if (op.cls_mode == 2) { i = c % op.nx; j = c / op.nx; }
    const Col<double> col = make_col(op, i, j);
    // a face whose neighbour is the column itself (one cell across a periodic
    // axis) couples the column to itself and is not part of its block
    const double musum = ((col.ce != col.c ? col.me : 0.0) + (col.cw != col.c ? col.mw : 0.0)) +
                         ((col.cn != col.c ? col.mn : 0.0) + (col.cs != col.c ? col.ms : 0.0));
    double e = 0.0, wprev = 0.0, dprev = 1.0;
    for (int k = 0; k < op.nz; ++k) {
        const double s = col.area * op.mass[k] + op.dk[k] * musum;
        const double w = col.area * op.wv[k];
        e = (k == 0) ? s : s + wprev * (e / dprev);
        const double d = w + e;
        fg[(long long)k * op.ncls + c] = 1.0 / d;
        fe[(long long)k * op.ncls + c] = e;
        if (fc) fc[(long long)k * op.ncls + c] = w / d;
        wprev = w;
        dprev = d;
    }
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) b[i] = (float)a[i];
}

}  // namespace pcg
