// libgbcg: conjugate gradient on a CSR matrix, one persistent cooperative
// kernel per solve on a GB300 (sm_103a), behind the C ABI of gbcg.h.
//
// The iteration is the CG recurrence of the textbook the paper cites for the
// method (Section IV): q = A p, alpha = rho / p.q, x += alpha p, r -= alpha q,
// stop when ||r|| <= tol ||b||, z = M^-1 r, beta = r.z / rho, p = z + beta p.
// One iteration is one SpMV, two dot products and three axpys (Table I's
// flop count, 2 NNZ + 10 N).  On GB300 the FP64 pipe (about 2 FMA per clock
// per SM) bounds this path before HBM does, so every phase does exactly the
// FP64 operations of the recurrence and nothing more:
//
//   phase A  p = z + beta p and q = A z + beta q over this CTA's rows (the
//            SpMV gathers z, streamed by TMA per warp; A p = A z + beta A p_old),
//            partial p.q                                  -> grid barrier
//   phase B  x += alpha p, r -= alpha q, z = dinv r (published for the
//            next SpMV), partial r.r and r.z              -> grid barrier
//            every CTA takes the same stop decision
//
// Two grid barriers per iteration: the direction p is only ever needed on
// the rows a thread owns, so it is updated inside phase A instead of in a
// phase of its own.
//
// Scalars never leave the device; sums are fixed-order (bitwise
// reproducible from run to run).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "cg_device.cuh"
#include "gbcg.h"
#include "handle.h"
#include "lowprec.h"
#include "plan.h"
#include "sellsolve.cuh"

using namespace gbcg;

static_assert(sizeof(I4) == sizeof(int4), "tile descriptor layout");

namespace {

// ------------------------------------------------------------ row state
// With RPT > 0 every thread keeps the vector entries of the rows it owns
// (lane l of warp w owns row r0 + l of each of the warp's tiles) in
// registers for the whole solve: x, r, z, p, q and 1/diag never round-trip
// through memory; only p is published (the SpMV gathers it) and x is written
// at the end.  RPT = 0 keeps every vector in global memory.
template <int RPT>
struct RegRows {
    int row[RPT > 0 ? RPT : 1];
    double x[RPT > 0 ? RPT : 1], r[RPT > 0 ? RPT : 1], z[RPT > 0 ? RPT : 1];
    double p[RPT > 0 ? RPT : 1], q[RPT > 0 ? RPT : 1], dinv[RPT > 0 ? RPT : 1];
};

// ------------------------------------------------------------ epilogues
struct EpiSetup {       // r = b - A x0, z = M^-1 r (gathered), p = z, q = 0; sums r.r, r.z, b.b
    const double *b;
    double *r;
    double *z;
    double *p;          // gathered copy of z
    double *pd;         // direction
    double *q;
    const double *dinv;
    int precond;
    double rr = 0.0, rz = 0.0, bb = 0.0;
    __device__ __forceinline__ void row(int i, double ax, int) {
        const double bi = b[i];
        const double ri = bi - ax;
        r[i] = ri;
        double zi = ri;
        if (precond) {
            zi = dinv[i] * ri;
            z[i] = zi;
        }
        p[i] = zi;
        pd[i] = zi;
        q[i] = 0.0;
        rr = fma(ri, ri, rr);
        rz = fma(ri, zi, rz);
        bb = fma(bi, bi, bb);
    }
};

template <int RPT>
struct RegSetup {       // the same, into registers (p is also published)
    RegRows<RPT> &R;
    const double *b;
    double *p;
    int precond;
    double rr = 0.0, rz = 0.0, bb = 0.0;
    __device__ __forceinline__ void row(int i, double ax, int j) {
        const double bi = b[i];
        const double ri = bi - ax;
        const double zi = precond ? R.dinv[j] * ri : ri;
        R.r[j] = ri;
        R.z[j] = zi;
        R.p[j] = zi;
        R.q[j] = 0.0;
        p[i] = zi;
        rr = fma(ri, ri, rr);
        rz = fma(ri, zi, rz);
        bb = fma(bi, bi, bb);
    }
};

struct EpiIter {        // p = z + beta p, q = A z + beta q; sum p . q
    double *q;
    double *pd;
    const double *z;    // the gathered vector (own rows read back)
    double beta;
    double pq = 0.0;
    double zi_ = 0.0, qi_ = 0.0, pi_ = 0.0;   // the row's entries, loaded ahead
    __device__ __forceinline__ void prefetch(int i) {
        zi_ = z[i];
        qi_ = q[i];
        pi_ = pd[i];
    }
    __device__ __forceinline__ void row(int i, double az, int) {
        const double qi = fma(beta, qi_, az);
        const double pi = fma(beta, pi_, zi_);
        q[i] = qi;
        pd[i] = pi;
        pq = fma(pi, qi, pq);
    }
};

template <int RPT>
struct RegIter {
    RegRows<RPT> &R;
    double beta;
    double pq = 0.0;
    __device__ __forceinline__ void row(int, double az, int j) {
        const double qi = fma(beta, R.q[j], az);
        const double pi = fma(beta, R.p[j], R.z[j]);
        R.q[j] = qi;
        R.p[j] = pi;
        pq = fma(pi, qi, pq);
    }
};

struct EpiTrue {        // sum (b - A x)^2
    const double *b;
    double acc = 0.0;
    __device__ __forceinline__ void row(int i, double ax, int) {
        const double t = b[i] - ax;
        acc = fma(t, t, acc);
    }
};

struct EpiStore {       // y = A x
    double *y;
    __device__ __forceinline__ void row(int i, double ax, int) { y[i] = ax; }
};

// Decisions thread 0 takes from the reduced scalars and broadcasts.
// Each slot is rewritten only after a __syncthreads that follows every read
// of its previous value.
constexpr int kCtlRun = 0;       // 1: continue iterating
constexpr int kCtlZeroB = 2;     // 1: b = 0, so x = 0
constexpr int kCtlTrue = 3;      // 1: compute the true residual

// ------------------------------------------------------- the solve kernel
// Scalar recurrences (alpha, beta, the stop test) run in thread 0 only: on
// GB300 an FP64 divide or square root executed by every warp would cost the
// FP64 pipe as much as a tile of the SpMV.
template <int RPT>
__global__ void __launch_bounds__(kThreads, 1) cg_solve_kernel(Params P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Smem S = carve_smem(smem_raw);
    init_pipeline(S);
    unsigned int epoch = 0;
    Pipe pipe;
    int set = 0;
    const int tid = threadIdx.x;
    const int row_lo = P.cta_row[blockIdx.x];
    const int row_hi = P.cta_row[blockIdx.x + 1];
    double *const p = P.p0;

    // thread 0's scalar state
    int status = CG_OK, iters = 0;
    double rr = 0.0, bb = 0.0, true_rr = -1.0, rho = 0.0, bnorm = 0.0;
    RegRows<RPT> R;
    if constexpr (RPT > 0) {
        const int t0 = P.cta_tile[blockIdx.x], nt = P.cta_tile[blockIdx.x + 1] - t0;
        const int w = tid >> 5, lane = tid & 31;
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            R.row[j] = -1;
            R.x[j] = 0.0;
            R.dinv[j] = 1.0;
            const int t = w + kWarps * j;
            if (t < nt) {
                const TileDesc d = load_desc(P, t0 + t);
                const int row = d.r0 + lane;
                if (row < d.r1) {
                    R.row[j] = row;
                    R.x[j] = P.x[row];
                    if (P.precond) R.dinv[j] = P.dinv[row];
                }
            }
        }
    }

    // ---- setup: r0 = b - A x0, z0 = M^-1 r0, p0 = z0; r.r, r.z, b.b
    bool run;
    {
        double v[3];
        if constexpr (RPT > 0) {
            RegSetup<RPT> epi{R, P.b, p, P.precond};
            if (!spmv_tiles<RPT, double, double, double>(P, S, pipe, P.vals, P.x, epi)) goto out;
            v[0] = epi.rr; v[1] = epi.rz; v[2] = epi.bb;
        } else {
            EpiSetup epi{P.b, P.r, P.z, p, P.pd, P.q, P.dinv, P.precond};
            if (!spmv_tiles<0, double, double, double>(P, S, pipe, P.vals, P.x, epi)) goto out;
            v[0] = epi.rr; v[1] = epi.rz; v[2] = epi.bb;
        }
        block_sum<3>(v, S);
        publish_partials<3>(P, set, v);
        if (!grid_barrier(P, epoch, S)) goto out;
        double tot[3];
        grid_totals<3>(P, set, tot);
        set ^= 1;
        if (tid == 0) {
            rr = tot[0];
            bb = tot[2];
            rho = tot[1];
            bnorm = sqrt(bb);
            int go = 0, zero_b = 0;
            if (!finite_bits(bb)) {
                status = CG_ENAN;
            } else if (bnorm == 0.0) {
                rr = 0.0;
                zero_b = 1;
            } else if (!finite_bits(rr) || !finite_bits(rho)) {
                status = CG_ENAN;
            } else if (sqrt(rr) <= P.tol * bnorm) {
                status = CG_OK;
            } else if (!(rho > 0.0)) {
                status = CG_EBREAKDOWN;
            } else {
                go = 1;
            }
            S.ctl[kCtlRun] = go;
            S.ctl[kCtlZeroB] = zero_b;
        }
        __syncthreads();
        run = S.ctl[kCtlRun] != 0;
        if (S.ctl[kCtlZeroB]) {  // b = 0: the solution is x = 0
            if constexpr (RPT > 0) {
#pragma unroll
                for (int j = 0; j < RPT; ++j) R.x[j] = 0.0;
            } else {
                for (int i = row_lo + tid; i < row_hi; i += kThreads) P.x[i] = 0.0;
            }
        }
    }

    // ---- the CG loop
    if (run) {
        if (tid == 0) status = CG_ENOCONV;
        double beta = 0.0;  // p_1 = z_0 and q_1 = A z_0
        for (int k = 1; k <= P.maxit; ++k) {
            // phase A: p = z + beta p, q = A z + beta q (= A p), p . q
            double pq;
            if constexpr (RPT > 0) {
                RegIter<RPT> ei{R, beta};
                if (!spmv_tiles<RPT, double, double, double>(P, S, pipe, P.vals, p, ei)) goto out;
                pq = ei.pq;
            } else {
                EpiIter ei{P.q, P.pd, p, beta};
                if (!spmv_tiles<0, double, double, double>(P, S, pipe, P.vals, p, ei)) goto out;
                pq = ei.pq;
            }
            double v1[1] = {pq};
            block_sum<1>(v1, S);
            publish_partials<1>(P, set, v1);
            if (!grid_barrier(P, epoch, S)) goto out;
            double sg[1];
            grid_totals<1>(P, set, sg);
            set ^= 1;
            if (tid == 0) {
                const double sigma = sg[0];
                int go = 0;
                if (!finite_bits(sigma)) status = CG_ENAN;
                else if (!(sigma > 0.0)) status = CG_EBREAKDOWN;
                else go = 1;
                S.bcast[0] = go ? rho / sigma : 0.0;
                S.ctl[kCtlRun] = go;
            }
            __syncthreads();
            if (!S.ctl[kCtlRun]) break;
            const double alpha = S.bcast[0];

            // phase B: x += alpha p, r -= alpha q, z = dinv r (published for
            // the next SpMV: every gather of phase A is over); r.r, r.z
            double prr = 0.0, prz = 0.0;
            if constexpr (RPT > 0) {
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    if (R.row[j] >= 0) {
                        R.x[j] = fma(alpha, R.p[j], R.x[j]);
                        const double ri = fma(-alpha, R.q[j], R.r[j]);
                        R.r[j] = ri;
                        prr = fma(ri, ri, prr);
                        double zi = ri;
                        if (P.precond) {
                            zi = R.dinv[j] * ri;
                            prz = fma(ri, zi, prz);
                        }
                        R.z[j] = zi;
                        p[R.row[j]] = zi;
                    }
                }
            } else {
                for (int i = row_lo + tid; i < row_hi; i += kThreads) {
                    const double pi = P.pd[i], qi = P.q[i], xi = P.x[i], ri0 = P.r[i];
                    P.x[i] = fma(alpha, pi, xi);
                    const double ri = fma(-alpha, qi, ri0);
                    P.r[i] = ri;
                    prr = fma(ri, ri, prr);
                    double zi = ri;
                    if (P.precond) {
                        zi = P.dinv[i] * ri;
                        prz = fma(ri, zi, prz);
                    }
                    p[i] = zi;
                }
            }
            double t2[2];
            if (P.precond) {
                double v2[2] = {prr, prz};
                block_sum<2>(v2, S);
                publish_partials<2>(P, set, v2);
                if (!grid_barrier(P, epoch, S)) goto out;
                grid_totals<2>(P, set, t2);
            } else {
                double v2[1] = {prr};
                block_sum<1>(v2, S);
                publish_partials<1>(P, set, v2);
                if (!grid_barrier(P, epoch, S)) goto out;
                double t1[1];
                grid_totals<1>(P, set, t1);
                t2[0] = t1[0];
                t2[1] = t1[0];
            }
            set ^= 1;
            if (tid == 0) {
                iters = k;
                rr = t2[0];
                const double rho_new = t2[1];
                int go = 0;
                if (!finite_bits(rr)) status = CG_ENAN;
                else if (sqrt(rr) <= P.tol * bnorm) status = CG_OK;
                else if (!finite_bits(rho_new)) status = CG_ENAN;
                else if (!(rho_new > 0.0)) status = CG_EBREAKDOWN;
                else if (k < P.maxit) go = 1;  // else ENOCONV: no further direction needed
                if (go) {
                    S.bcast[1] = rho_new / rho;
                    rho = rho_new;
                }
                S.ctl[kCtlRun] = go;
            }
            __syncthreads();
            if (!S.ctl[kCtlRun]) break;
            beta = S.bcast[1];
        }
    }

    // ---- publish x (register mode), then the true residual ||b - A x||
    if constexpr (RPT > 0) {
#pragma unroll
        for (int j = 0; j < RPT; ++j)
            if (R.row[j] >= 0) P.x[R.row[j]] = R.x[j];
    }
    {
        if (tid == 0) S.ctl[kCtlTrue] = (P.true_res && status != CG_ENAN && bb != 0.0) ? 1 : 0;
        __syncthreads();
        const bool want_true = S.ctl[kCtlTrue] != 0;
        if (tid == 0 && P.true_res && status != CG_ENAN && bb == 0.0) true_rr = 0.0;
        if (want_true) {
            if constexpr (RPT > 0) {
                if (!grid_barrier(P, epoch, S)) goto out;  // every x entry is written
            }
            EpiTrue et{P.b};
            if (!spmv_tiles<RPT, double, double, double>(P, S, pipe, P.vals, P.x, et)) goto out;
            double v[1] = {et.acc};
            block_sum<1>(v, S);
            publish_partials<1>(P, set, v);
            if (!grid_barrier(P, epoch, S)) goto out;
            double t[1];
            grid_totals<1>(P, set, t);
            if (tid == 0) true_rr = t[0];
        }
    }

    if (blockIdx.x == 0 && tid == 0) {
        P.st->iters = iters;
        P.st->rr = rr;
        P.st->bb = bb;
        P.st->true_rr = true_rr;
        atomicCAS(&P.st->status, 0, status);
    }
out:
    drain<double, double>(P, S, pipe, p);
}

// ------------------------------------------- the SELL-32 solve kernel
// For systems with at most 31 slices of 32 rows per SM (n <= 150,784 on 152
// SMs): 1024 threads per CTA.  Warp 0 is the control warp and owns no slice;
// warp w >= 1 of CTA c owns slice cut[c] + w - 1 (contiguous ranges balanced
// by FP64 work on the host) and lane l its row, whose x, r, z, p, q and
// 1/diag stay in registers.  The SpMV reads the SELL-32 copy straight from L2
// (every load coalesced), so no warp waits for a shared-memory stage and
// every warp has at most one slice.
//
// Two grid barriers per iteration, as in cg_solve_kernel, with one change of
// order: the SpMV A z of iteration k+1 needs only z, so it starts as soon as
// the barrier that publishes z has passed, and the control warp meanwhile
// adds the grid totals of r.r and r.z, takes the stop decision and forms
// beta = rho'/rho.  The warps then finish q = A z + beta q and p = z + beta p
// (the last iteration's SpMV is computed and dropped).
constexpr int kSliceMaxPerCta = kSellSolveThreads / 32 - 1;   // warps 1..31
constexpr int kSliceVecCost = 8;   // FP64 vector operations per row, in SpMV-width units

template <bool PRE>
__global__ void __launch_bounds__(kSellSolveThreads, 1)
    cg_sell_kernel(Params P, SellMatrix M, const int32_t *__restrict__ cut) {
    __shared__ double red[3 * kSellSolveThreads];
    __shared__ double quarter[12];
    __shared__ double bcast[8];
    __shared__ int ctl[16];
    __shared__ long long slice_a[kSellSolveThreads / 32];
    __shared__ int slice_w[kSellSolveThreads / 32];
    Smem S{};
    S.red = red;
    S.bcast = bcast;
    S.ctl = ctl;
    unsigned int epoch = 0;
    int set = 0;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int t = cut[blockIdx.x] + w - 1;
    const bool has_slice = w >= 1 && t < cut[blockIdx.x + 1];   // uniform over the warp; never warp 0
    const int row = t * 32 + lane;
    const bool own = has_slice && row < P.n;
    double *const zg = P.p0;   // z, gathered by the SpMV

    // thread 0's scalar state
    int status = CG_OK, iters = 0;
    double rr = 0.0, bb = 0.0, true_rr = -1.0, rho = 0.0, bnorm = 0.0, tol2bb = 0.0;
    // the row's vectors
    double x = own ? P.x[row] : 0.0, r = 0.0, z = 0.0, p = 0.0, q = 0.0;
    // 1/diag is read from memory (L1) where it is used: a register for it
    // makes the Jacobi instantiation spill
    const double *__restrict__ dinv_g = P.dinv;

    // ---- setup: r0 = b - A x0, z0 = M^-1 r0, p0 = z0; r.r, r.z, b.b
    bool run;
    {
        const double ax = has_slice ? sell_slice_sum(M, t, P.x, 0.0) : 0.0;
        double v[3] = {0.0, 0.0, 0.0};
        if (own) {
            const double bi = P.b[row];
            r = bi - ax;
            z = PRE ? __ldg(dinv_g + row) * r : r;
            p = z;
            zg[row] = z;
            v[0] = r * r;
            v[1] = r * z;
            v[2] = bi * bi;
        }
        block_sum_1k<3>(v, red, quarter);
        publish_partials<3>(P, set, v);
        if (!grid_barrier<false>(P, epoch, S)) goto out;
        double tot[3];
        grid_totals_1k<3>(P, set, tot, quarter);
        set ^= 1;
        if (tid == 0) {
            rr = tot[0];
            bb = tot[2];
            rho = tot[1];
            bnorm = sqrt(bb);
            tol2bb = (P.tol * bnorm) * (P.tol * bnorm);
            int go = 0, zero_b = 0;
            if (!finite_bits(bb)) {
                status = CG_ENAN;
            } else if (bnorm == 0.0) {
                rr = 0.0;
                zero_b = 1;
            } else if (!finite_bits(rr) || !finite_bits(rho)) {
                status = CG_ENAN;
            } else if (rr <= tol2bb) {
                status = CG_OK;
            } else if (!(rho > 0.0)) {
                status = CG_EBREAKDOWN;
            } else {
                go = 1;
            }
            ctl[kCtlRun] = go;
            ctl[kCtlZeroB] = zero_b;
        }
        __syncthreads();
        run = ctl[kCtlRun] != 0;
        if (ctl[kCtlZeroB]) x = 0.0;  // b = 0: the solution is x = 0
    }

    // ---- the CG loop
    if (run) {
        if (tid == 0) status = CG_ENOCONV;
        constexpr int NB = PRE ? 2 : 1;
        // thread 0: decision on the r.r, r.z totals of iteration kk (recorded
        // in kk's exchange); go = 1 sets beta for the next iteration
        auto decide = [&](int kk, const double (&t2)[NB]) {
            iters = kk;
            rr = t2[0];
            const double rho_new = t2[NB - 1];
            int go = 0;
            if (!finite_bits(rr)) status = CG_ENAN;
            else if (rr <= tol2bb) status = CG_OK;
            else if (!finite_bits(rho_new)) status = CG_ENAN;
            else if (!(rho_new > 0.0)) status = CG_EBREAKDOWN;
            else if (kk < P.maxit) go = 1;  // else ENOCONV
            if (go) {
                bcast[1] = rho_new / rho;
                rho = rho_new;
            }
            ctl[kCtlRun] = go;
        };
        // each slice's entries in this CTA's own rows come first (k < wl); the
        // first iteration's are added here, the others' while the barrier
        // that publishes z completes
        const int wl = has_slice ? (M.split ? M.split[t] : 0) : 0;
        // the slice's first entry and width, loaded once for the whole solve
        // and kept in shared memory (registers are at the 64 of 1024 threads)
        if (lane == 0 && has_slice) {
            slice_a[w] = M.ptr[t];
            slice_w[w] = (int)((M.ptr[t + 1] - slice_a[w]) >> 5);
        }
        __syncwarp();
        double azl = has_slice ? sell_slice_sum_at(M, t, slice_a[w], slice_w[w], zg, 0.0, 0, wl) : 0.0;
        for (int k = 1;; ++k) {
            // phase A: az = A z on warps 1..31 (the rest of each row, from
            // azl); the control warp decides on iteration k-1 meanwhile
            const double az = has_slice ? sell_slice_sum_at(M, t, slice_a[w], slice_w[w], zg, azl, wl) : 0.0;
            if (k > 1 && w == 0) {
                double t2[NB];
                grid_totals<NB>(P, set ^ 1, t2);
                if (tid == 0) decide(k - 1, t2);
            }
            __syncthreads();
            if (k > 1 && !ctl[kCtlRun]) break;
            const double beta = k > 1 ? bcast[1] : 0.0;
            // p = z + beta p, q = A z + beta q (= A p), p . q
            double v1[1] = {0.0};
            if (own) {
                q = fma(beta, q, az);
                p = fma(beta, p, z);
                v1[0] = p * q;
            }
            block_sum_1k<1>(v1, red, quarter);
            publish_partials<1>(P, set, v1);
            if (!grid_barrier<false>(P, epoch, S)) goto out;
            double sg[1];
            grid_totals_1k<1>(P, set, sg, quarter);
            set ^= 1;
            if (tid == 0) {
                const double sigma = sg[0];
                int go = 0;
                if (!finite_bits(sigma)) status = CG_ENAN;
                else if (!(sigma > 0.0)) status = CG_EBREAKDOWN;
                else go = 1;
                bcast[0] = go ? rho / sigma : 0.0;
                ctl[kCtlRun] = go;
            }
            __syncthreads();
            if (!ctl[kCtlRun]) break;
            const double alpha = bcast[0];

            // phase B: r -= alpha q, z = dinv r (published); r.r, r.z (plain
            // CG: z = r and r.z = r.r, one sum); x += alpha p below
            double v2[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) v2[j] = 0.0;
            if (own) {
                r = fma(-alpha, q, r);
                z = PRE ? __ldg(dinv_g + row) * r : r;
                zg[row] = z;
                v2[0] = r * r;
                if constexpr (PRE) v2[NB - 1] = r * z;
            }
            block_sum_1k<NB>(v2, red, quarter);
            publish_partials<NB>(P, set, v2);
            // the barrier that publishes z: the warps with a slice add its
            // entries in this CTA's own rows (z written before grid_arrive's
            // __syncthreads) while thread 0 waits for the other CTAs
            grid_arrive(P, epoch);
            if (has_slice) {
                // x is read by nothing before the end: x += alpha p leaves
                // the critical path (p changes only in the next phase A)
                if (own) x = fma(alpha, p, x);
                azl = sell_slice_sum_at(M, t, slice_a[w], slice_w[w], zg, 0.0, 0, wl);
            } else if (tid == 0) {
                ctl[15] = grid_wait<false>(P, epoch);
            }
            __syncthreads();
            if (!ctl[15]) goto out;
            set ^= 1;   // this exchange's partials are set ^ 1 from here on
            if (k == P.maxit) {   // the last allowed iteration: decide now
                if (w == 0) {
                    double t2[NB];
                    grid_totals<NB>(P, set ^ 1, t2);
                    if (tid == 0) decide(k, t2);
                }
                __syncthreads();
                break;
            }
        }
    }

    // ---- publish x, then the true residual ||b - A x||
    if (own) P.x[row] = x;
    {
        if (tid == 0) ctl[kCtlTrue] = (P.true_res && status != CG_ENAN && bb != 0.0) ? 1 : 0;
        __syncthreads();
        const bool want_true = ctl[kCtlTrue] != 0;
        if (tid == 0 && P.true_res && status != CG_ENAN && bb == 0.0) true_rr = 0.0;
        if (want_true) {
            if (!grid_barrier<false>(P, epoch, S)) goto out;  // every x entry is written
            const double ax = has_slice ? sell_slice_sum(M, t, P.x, 0.0) : 0.0;
            double v[1] = {0.0};
            if (own) {
                const double d = P.b[row] - ax;
                v[0] = d * d;
            }
            block_sum_1k<1>(v, red, quarter);
            publish_partials<1>(P, set, v);
            if (!grid_barrier<false>(P, epoch, S)) goto out;
            double tt[1];
            grid_totals_1k<1>(P, set, tt, quarter);
            if (tid == 0) true_rr = tt[0];
        }
    }

    if (blockIdx.x == 0 && tid == 0) {
        P.st->iters = iters;
        P.st->rr = rr;
        P.st->bb = bb;
        P.st->true_rr = true_rr;
        atomicCAS(&P.st->status, 0, status);
    }
out:
    return;
}

// ------------------------------------------ the SELL-32 memory-mode solve
// For systems with more slices than the slice kernel holds (n > 150,784 on
// 152 SMs): the same CG iteration with the vectors in global memory.  The
// vectors (x, r, p, q, the published z, 1/diag: 6 x 8 bytes per row) stay in
// L2 while the matrix streams through it marked evict-first.  Warp w of CTA
// c takes slices cut[c] + w, + 32, ... of the CTA's contiguous range (ranges
// balanced by FP64 work on the host); a row is always read and written by
// the same thread.  Two grid barriers per iteration; each decision is taken
// before the next phase starts.

template <bool PRE>
__global__ void __launch_bounds__(kSellSolveThreads, 1)
    cg_sellmem_kernel(Params P, SellMatrix M, const int32_t *__restrict__ cut) {
    __shared__ double red[3 * kSellSolveThreads];
    __shared__ double quarter[12];
    __shared__ double bcast[8];
    __shared__ int ctl[16];
    Smem S{};
    S.red = red;
    S.bcast = bcast;
    S.ctl = ctl;
    unsigned int epoch = 0;
    int set = 0;
    constexpr int kW = kSellSolveThreads / 32;
    const int tid = threadIdx.x, lane = tid & 31;
    const int t0 = cut[blockIdx.x] + (tid >> 5), t1 = cut[blockIdx.x + 1];
    double *const zg = P.p0;   // z: the vector the SpMV gathers
    double *const pv = P.pd;   // p

    // thread 0's scalar state
    int status = CG_OK, iters = 0;
    double rr = 0.0, bb = 0.0, true_rr = -1.0, rho = 0.0, bnorm = 0.0, tol2bb = 0.0;

    // ---- setup: r0 = b - A x0, z0 = M^-1 r0, p0 = z0, q = 0; r.r, r.z, b.b
    bool run;
    {
        double v[3] = {0.0, 0.0, 0.0};
        for (int t = t0; t < t1; t += kW) {
            const double ax = sell_slice_sum<kSellUnrollMem>(M, t, P.x, 0.0);
            const int row = t * 32 + lane;
            if (row < P.n) {
                const double bi = P.b[row];
                const double ri = bi - ax;
                const double zi = PRE ? __ldg(P.dinv + row) * ri : ri;
                P.r[row] = ri;
                zg[row] = zi;
                pv[row] = zi;
                P.q[row] = 0.0;
                v[0] = fma(ri, ri, v[0]);
                v[1] = fma(ri, zi, v[1]);
                v[2] = fma(bi, bi, v[2]);
            }
        }
        block_sum_1k<3>(v, red, quarter);
        publish_partials<3>(P, set, v);
        if (!grid_barrier<false>(P, epoch, S)) goto out;
        double tot[3];
        grid_totals_1k<3>(P, set, tot, quarter);
        set ^= 1;
        if (tid == 0) {
            rr = tot[0];
            bb = tot[2];
            rho = tot[1];
            bnorm = sqrt(bb);
            tol2bb = (P.tol * bnorm) * (P.tol * bnorm);
            int go = 0, zero_b = 0;
            if (!finite_bits(bb)) {
                status = CG_ENAN;
            } else if (bnorm == 0.0) {
                rr = 0.0;
                zero_b = 1;
            } else if (!finite_bits(rr) || !finite_bits(rho)) {
                status = CG_ENAN;
            } else if (rr <= tol2bb) {
                status = CG_OK;
            } else if (!(rho > 0.0)) {
                status = CG_EBREAKDOWN;
            } else {
                go = 1;
            }
            ctl[kCtlRun] = go;
            ctl[kCtlZeroB] = zero_b;
        }
        __syncthreads();
        run = ctl[kCtlRun] != 0;
        if (ctl[kCtlZeroB])   // b = 0: the solution is x = 0
            for (int t = t0; t < t1; t += kW)
                if (t * 32 + lane < P.n) P.x[t * 32 + lane] = 0.0;
    }

    // ---- the CG loop
    if (run) {
        if (tid == 0) status = CG_ENOCONV;
        constexpr int NB = PRE ? 2 : 1;
        double beta = 0.0;   // p_1 = z_0, q_1 = A z_0
        for (int k = 1; k <= P.maxit; ++k) {
            // phase A: q = A z + beta q (= A p), p = z + beta p; p . q
            double v1[1] = {0.0};
            for (int t = t0; t < t1; t += kW) {
                const double az = sell_slice_sum<kSellUnrollMem>(M, t, zg, 0.0);
                const int row = t * 32 + lane;
                if (row < P.n) {
                    const double qi = fma(beta, P.q[row], az);
                    const double pi = fma(beta, pv[row], zg[row]);
                    P.q[row] = qi;
                    pv[row] = pi;
                    v1[0] = fma(pi, qi, v1[0]);
                }
            }
            block_sum_1k<1>(v1, red, quarter);
            publish_partials<1>(P, set, v1);
            if (!grid_barrier<false>(P, epoch, S)) goto out;
            double sg[1];
            grid_totals_1k<1>(P, set, sg, quarter);
            set ^= 1;
            if (tid == 0) {
                const double sigma = sg[0];
                int go = 0;
                if (!finite_bits(sigma)) status = CG_ENAN;
                else if (!(sigma > 0.0)) status = CG_EBREAKDOWN;
                else go = 1;
                bcast[0] = go ? rho / sigma : 0.0;
                ctl[kCtlRun] = go;
            }
            __syncthreads();
            if (!ctl[kCtlRun]) break;
            const double alpha = bcast[0];

            // phase B: x += alpha p, r -= alpha q, z = dinv r (published); r.r, r.z
            double v2[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) v2[j] = 0.0;
            for (int t = t0; t < t1; t += kW) {
                const int row = t * 32 + lane;
                if (row < P.n) {
                    const double ri = fma(-alpha, P.q[row], P.r[row]);
                    P.x[row] = fma(alpha, pv[row], P.x[row]);
                    P.r[row] = ri;
                    const double zi = PRE ? __ldg(P.dinv + row) * ri : ri;
                    zg[row] = zi;
                    v2[0] = fma(ri, ri, v2[0]);
                    if constexpr (PRE) v2[NB - 1] = fma(ri, zi, v2[NB - 1]);
                }
            }
            block_sum_1k<NB>(v2, red, quarter);
            publish_partials<NB>(P, set, v2);
            if (!grid_barrier<false>(P, epoch, S)) goto out;
            double t2[NB];
            grid_totals_1k<NB>(P, set, t2, quarter);
            set ^= 1;
            if (tid == 0) {
                iters = k;
                rr = t2[0];
                const double rho_new = t2[NB - 1];
                int go = 0;
                if (!finite_bits(rr)) status = CG_ENAN;
                else if (rr <= tol2bb) status = CG_OK;
                else if (!finite_bits(rho_new)) status = CG_ENAN;
                else if (!(rho_new > 0.0)) status = CG_EBREAKDOWN;
                else if (k < P.maxit) go = 1;  // else ENOCONV
                if (go) {
                    bcast[1] = rho_new / rho;
                    rho = rho_new;
                }
                ctl[kCtlRun] = go;
            }
            __syncthreads();
            if (!ctl[kCtlRun]) break;
            beta = bcast[1];
        }
    }

    // ---- the true residual ||b - A x||
    {
        if (tid == 0) ctl[kCtlTrue] = (P.true_res && status != CG_ENAN && bb != 0.0) ? 1 : 0;
        __syncthreads();
        const bool want_true = ctl[kCtlTrue] != 0;
        if (tid == 0 && P.true_res && status != CG_ENAN && bb == 0.0) true_rr = 0.0;
        if (want_true) {
            if (!grid_barrier<false>(P, epoch, S)) goto out;  // every x entry is written
            double v[1] = {0.0};
            for (int t = t0; t < t1; t += kW) {
                const double ax = sell_slice_sum<kSellUnrollMem>(M, t, P.x, 0.0);
                const int row = t * 32 + lane;
                if (row < P.n) {
                    const double d = P.b[row] - ax;
                    v[0] = fma(d, d, v[0]);
                }
            }
            block_sum_1k<1>(v, red, quarter);
            publish_partials<1>(P, set, v);
            if (!grid_barrier<false>(P, epoch, S)) goto out;
            double tt[1];
            grid_totals_1k<1>(P, set, tt, quarter);
            if (tid == 0) true_rr = tt[0];
        }
    }

    if (blockIdx.x == 0 && tid == 0) {
        P.st->iters = iters;
        P.st->rr = rr;
        P.st->bb = bb;
        P.st->true_rr = true_rr;
        atomicCAS(&P.st->status, 0, status);
    }
out:
    return;
}

// ---------------------------------------------- mixed-precision solve
// Iterative refinement: the outer loop keeps x and the residual in FP64 with
// the FP64 matrix (r = b - A x, stop when ||r|| <= tol ||b||, x += d); each
// correction d solves A_lo d = r by CG in FP32 (FP32 vectors, FP32 products
// and per-thread sums) on the low-precision copy of A (FP32 or BF16
// off-diagonals plus the compensated FP32 diagonal), optionally with Jacobi,
// until its residual falls by inner_tol.  One persistent launch runs it all.
struct EpiOuter {       // r = b - A x; inner start: r32, z32 = M r32 (gathered copy in p32),
                        // direction pd32 = z32, q32 = 0, d32 = 0
    const double *b;
    float *r32, *p32, *pd32, *q32, *d32;
    const float *dinv32;
    int precond;
    double rr = 0.0, bb = 0.0;
    float rz = 0.0f;
    __device__ __forceinline__ void row(int i, double ax, int) {
        const double bi = b[i];
        const double ri = bi - ax;
        rr = fma(ri, ri, rr);
        bb = fma(bi, bi, bb);
        const float rf = (float)ri;
        r32[i] = rf;
        const float zf = precond ? dinv32[i] * rf : rf;
        p32[i] = zf;
        pd32[i] = zf;
        q32[i] = 0.0f;
        d32[i] = 0.0f;
        rz = fmaf(rf, zf, rz);
    }
};

struct EpiInner {       // p = z + beta p, q = A_lo z + beta q (A_lo with its compensated diagonal); p . q
    float *q32;
    float *pd32;
    const float *z32;   // the gathered vector (own rows read back)
    const float *diag;
    float beta;
    float pq = 0.0f;
    float zi_ = 0.0f, qi_ = 0.0f, pi_ = 0.0f, di_ = 0.0f;   // the row's entries, loaded ahead
    __device__ __forceinline__ void prefetch(int i) {
        zi_ = z32[i];
        qi_ = q32[i];
        pi_ = pd32[i];
        di_ = __ldg(diag + i);
    }
    __device__ __forceinline__ void row(int i, float s, int) {
        const float qi = fmaf(beta, qi_, fmaf(di_, zi_, s));
        const float pi = fmaf(beta, pi_, zi_);
        q32[i] = qi;
        pd32[i] = pi;
        pq = fmaf(pi, qi, pq);
    }
};

template <class VT>
__global__ void __launch_bounds__(kThreads, 1) cg_ir_kernel(Params P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Smem S = carve_smem(smem_raw);
    init_pipeline(S);
    unsigned int epoch = 0;
    Pipe pipe;
    int set = 0;
    const int tid = threadIdx.x;
    const int row_lo = P.cta_row[blockIdx.x];
    const int row_hi = P.cta_row[blockIdx.x + 1];
    const VT *vlo = nullptr;
    if constexpr (sizeof(VT) == 4) vlo = reinterpret_cast<const VT *>(P.vals32);
    else vlo = reinterpret_cast<const VT *>(P.vals16);

    // thread 0's scalar state
    int status = CG_ENOCONV, inner_total = 0, outer = 0;
    double rr = 0.0, bb = 0.0, bnorm = 0.0;

    for (int o = 0;; ++o) {
        // ---- outer residual in FP64 and the start of the inner solve
        double rho;
        {
            EpiOuter eo{P.b, P.r32, P.p32, P.pd32, P.q32, P.d32, P.dinv32, P.precond};
            if (!spmv_tiles<0, double, double, double>(P, S, pipe, P.vals, P.x, eo, true)) goto out;
            double v[3] = {eo.rr, eo.bb, (double)eo.rz};
            block_sum<3>(v, S);
            publish_partials<3>(P, set, v);
            if (!grid_barrier(P, epoch, S)) goto out;
            double t[3];
            grid_totals<3>(P, set, t);
            set ^= 1;
            if (tid == 0) {
                rr = t[0];
                if (o == 0) {
                    bb = t[1];
                    bnorm = sqrt(bb);
                }
                int go = 0, zero_b = 0;
                if (!finite_bits(bb) || !finite_bits(rr) || !finite_bits(t[2])) status = CG_ENAN;
                else if (bnorm == 0.0) { status = CG_OK; zero_b = 1; rr = 0.0; }
                else if (sqrt(rr) <= P.tol * bnorm) status = CG_OK;
                else if (o == P.max_outer || inner_total >= P.maxit) status = CG_ENOCONV;
                else if (!(t[2] > 0.0)) status = CG_EBREAKDOWN;
                else go = 1;
                S.bcast[0] = t[2];                       // rho of the inner start
                S.bcast[1] = P.inner_tol * sqrt(t[0]) ;  // inner target on ||r32||
                S.ctl[kCtlRun] = go;
                S.ctl[kCtlZeroB] = zero_b;
            }
            __syncthreads();
            if (S.ctl[kCtlZeroB])
                for (int i = row_lo + tid; i < row_hi; i += kThreads) P.x[i] = 0.0;
            if (!S.ctl[kCtlRun]) break;
            rho = S.bcast[0];  // only thread 0 uses rho; the others never read it again
        }

        // ---- inner CG in FP32 on A_lo d = r (two barriers per iteration, as
        // in the FP64 solve: the SpMV gathers z and q = A z + beta q)
        float beta = 0.0f;
        for (int k = 1;; ++k) {
            EpiInner ei{P.q32, P.pd32, P.p32, P.diag_lo, beta};
            if (!spmv_tiles<0, VT, float, float>(P, S, pipe, vlo, P.p32, ei, true)) goto out;
            double v1[1] = {(double)ei.pq};
            block_sum<1>(v1, S);
            publish_partials<1>(P, set, v1);
            if (!grid_barrier(P, epoch, S)) goto out;
            double sg[1];
            grid_totals<1>(P, set, sg);
            set ^= 1;
            if (tid == 0) {
                int go = 1;
                if (!finite_bits(sg[0]) || !(sg[0] > 0.0)) go = 0;  // inner breakdown: keep d
                S.bcast[2] = go ? rho / sg[0] : 0.0;
                S.ctl[kCtlRun] = go;
                if (!go && k == 1) status = finite_bits(sg[0]) ? CG_EBREAKDOWN : CG_ENAN;
            }
            __syncthreads();
            if (!S.ctl[kCtlRun]) break;
            const float alpha = (float)S.bcast[2];
            float prr = 0.0f, prz = 0.0f;
            // four rows per thread at a time: every load of the four is issued
            // before the first store (the arrays do not alias)
            constexpr int kU = 4;
            for (int i0 = row_lo + tid; i0 < row_hi; i0 += kU * kThreads) {
                float pv[kU], qv[kU], dv[kU], rv[kU], iv[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int i = i0 + u * kThreads;
                    const bool in = i < row_hi;
                    pv[u] = in ? P.pd32[i] : 0.0f;
                    qv[u] = in ? P.q32[i] : 0.0f;
                    dv[u] = in ? P.d32[i] : 0.0f;
                    rv[u] = in ? P.r32[i] : 0.0f;
                    iv[u] = in && P.precond ? __ldg(P.dinv32 + i) : 1.0f;
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int i = i0 + u * kThreads;
                    if (i >= row_hi) break;
                    P.d32[i] = fmaf(alpha, pv[u], dv[u]);
                    const float ri = fmaf(-alpha, qv[u], rv[u]);
                    P.r32[i] = ri;
                    prr = fmaf(ri, ri, prr);
                    float zi = ri;
                    if (P.precond) {
                        zi = iv[u] * ri;
                        prz = fmaf(ri, zi, prz);
                    }
                    P.p32[i] = zi;   // gathered by the next SpMV (every gather of this one is over)
                }
            }
            double v2[2] = {(double)prr, (double)(P.precond ? prz : prr)};
            block_sum<2>(v2, S);
            publish_partials<2>(P, set, v2);
            if (!grid_barrier(P, epoch, S)) goto out;
            double t2[2];
            grid_totals<2>(P, set, t2);
            set ^= 1;
            if (tid == 0) {
                ++inner_total;
                int go = 0;
                const double rin = t2[0], rho_new = t2[1];
                if (!finite_bits(rin) || !finite_bits(rho_new) || !(rho_new > 0.0)) go = 0;
                else if (sqrt(rin) <= S.bcast[1]) go = 0;                 // inner target met
                else if (k >= P.max_inner || inner_total >= P.maxit) go = 0;
                else go = 1;
                if (go) {
                    S.bcast[3] = rho_new / rho;
                    rho = rho_new;
                }
                S.ctl[kCtlRun] = go;
            }
            __syncthreads();
            if (!S.ctl[kCtlRun]) break;
            beta = (float)S.bcast[3];
        }
        // ---- x += d in FP64
        for (int i = row_lo + tid; i < row_hi; i += kThreads) P.x[i] += (double)P.d32[i];
        if (tid == 0) outer = o + 1;
        if (!grid_barrier(P, epoch, S)) goto out;
    }

    if (blockIdx.x == 0 && tid == 0) {
        P.st->iters = inner_total;
        P.st->outer = outer;
        P.st->rr = rr;
        P.st->bb = bb;
        P.st->true_rr = rr;  // the outer residual is the true FP64 residual
        atomicCAS(&P.st->status, 0, status);
    }
out:
    drain<float, float>(P, S, pipe, P.p32);
}

// ------------------------------- mixed-precision solve on the SELL-32 copies
// The refinement of cg_ir_kernel (same outer FP64 residual, inner FP32 CG on
// A_lo d = r to inner_tol, x += d) with both SpMVs on SELL-32: the outer one
// on the FP64 copy, the inner one on a copy of the low-precision
// off-diagonals in the same layout (diagonal slots zero, the compensated
// FP32 diagonal kept apart).  The inner vectors are FP32 in memory
// (L2-resident: 28 bytes per row) and the matrix streams 6 (FP32) or 4
// (BF16) bytes per entry.  Warp w of CTA c takes slices cut[c] + w, + 32, ...
// of its CTA's range, as in cg_sellmem_kernel; a row is always read and
// written by the same thread.  Used for the systems of the slice kernel (at
// most 31 slices per CTA), where its iteration is the shorter one.
__device__ __forceinline__ float lo_load(const float *p, bool st) { return mload(p, st); }
__device__ __forceinline__ float lo_load(const __nv_bfloat16 *p, bool st) {
    const unsigned short u = st ? __ldcs(reinterpret_cast<const unsigned short *>(p))
                                : __ldcg(reinterpret_cast<const unsigned short *>(p));
    return __uint_as_float((unsigned int)u << 16);
}

// Row sum of lane's row in slice t with low-precision values, FP32 gathers
// (coherent L1 loads: x is written by this kernel) and FP32 accumulation.
// FP32 FMAs hide no latency here, so a batch keeps 18 entries in flight.
constexpr int kSellUnrollLo = 18;

template <class VT>
__device__ __forceinline__ float sell_slice_sum_lo(const SellMatrix &M, const VT *vlo, int t, const float *x) {
    const int lane = threadIdx.x & 31;
    const bool st = M.stream != 0;
    const long long a = M.ptr[t];
    const int w = (int)((M.ptr[t + 1] - a) >> 5);
    const int row = t * 32 + lane;
    const VT *vv = vlo + a + lane;
    float s0 = 0.0f, s1 = 0.0f;
    int k = 0;
    if (M.cols16) {
        const int16_t *cc = M.cols16 + a + lane;
        for (; k + kSellUnrollLo <= w; k += kSellUnrollLo) {
            float vr[kSellUnrollLo], xr[kSellUnrollLo];
#pragma unroll
            for (int u = 0; u < kSellUnrollLo; ++u) {
                vr[u] = lo_load(vv + (k + u) * 32, st);
                xr[u] = __ldca(x + bchk(row + (int)mload(cc + (k + u) * 32, st), M.n));
            }
#pragma unroll
            for (int u = 0; u < kSellUnrollLo; ++u) {
                if (u & 1) s1 = fmaf(vr[u], xr[u], s1);
                else s0 = fmaf(vr[u], xr[u], s0);
            }
        }
        for (; k < w; ++k) s0 = fmaf(lo_load(vv + k * 32, st), __ldca(x + bchk(row + (int)mload(cc + k * 32, st), M.n)), s0);
    } else {
        const int32_t *cc = M.cols32 + a + lane;
        for (; k + kSellUnrollLo <= w; k += kSellUnrollLo) {
            float vr[kSellUnrollLo], xr[kSellUnrollLo];
#pragma unroll
            for (int u = 0; u < kSellUnrollLo; ++u) {
                vr[u] = lo_load(vv + (k + u) * 32, st);
                xr[u] = __ldca(x + bchk(mload(cc + (k + u) * 32, st), M.n));
            }
#pragma unroll
            for (int u = 0; u < kSellUnrollLo; ++u) {
                if (u & 1) s1 = fmaf(vr[u], xr[u], s1);
                else s0 = fmaf(vr[u], xr[u], s0);
            }
        }
        for (; k < w; ++k) s0 = fmaf(lo_load(vv + k * 32, st), __ldca(x + bchk(mload(cc + k * 32, st), M.n)), s0);
    }
    return s0 + s1;
}

template <class VT>
__global__ void __launch_bounds__(kSellSolveThreads, 1)
    cg_irsell_kernel(Params P, SellMatrix M, const VT *__restrict__ vlo, const int32_t *__restrict__ cut) {
    __shared__ double red[3 * kSellSolveThreads];
    __shared__ double quarter[12];
    __shared__ double bcast[8];
    __shared__ int ctl[16];
    Smem S{};
    S.red = red;
    S.bcast = bcast;
    S.ctl = ctl;
    unsigned int epoch = 0;
    int set = 0;
    constexpr int kW = kSellSolveThreads / 32;
    const int tid = threadIdx.x, lane = tid & 31;
    const int t0 = cut[blockIdx.x] + (tid >> 5), t1 = cut[blockIdx.x + 1];

    // thread 0's scalar state
    int status = CG_ENOCONV, inner_total = 0, outer = 0;
    double rr = 0.0, bb = 0.0, bnorm = 0.0;

    for (int o = 0;; ++o) {
        // ---- outer residual in FP64 and the start of the inner solve
        double rho;
        {
            double v[3] = {0.0, 0.0, 0.0};   // r.r, b.b, r32.z32
            float rz = 0.0f;
            for (int t = t0; t < t1; t += kW) {
                const double ax = sell_slice_sum(M, t, P.x, 0.0);
                const int row = t * 32 + lane;
                if (row < P.n) {
                    const double bi = P.b[row];
                    const double ri = bi - ax;
                    v[0] = fma(ri, ri, v[0]);
                    v[1] = fma(bi, bi, v[1]);
                    const float rf = (float)ri;
                    const float zf = P.precond ? __ldg(P.dinv32 + row) * rf : rf;
                    P.r32[row] = rf;
                    P.p32[row] = zf;
                    P.pd32[row] = zf;
                    P.q32[row] = 0.0f;
                    P.d32[row] = 0.0f;
                    rz = fmaf(rf, zf, rz);
                }
            }
            v[2] = (double)rz;
            block_sum_1k<3>(v, red, quarter);
            publish_partials<3>(P, set, v);
            if (!grid_barrier<false>(P, epoch, S)) goto out;
            double tt[3];
            grid_totals_1k<3>(P, set, tt, quarter);
            set ^= 1;
            if (tid == 0) {
                rr = tt[0];
                if (o == 0) {
                    bb = tt[1];
                    bnorm = sqrt(bb);
                }
                int go = 0, zero_b = 0;
                if (!finite_bits(bb) || !finite_bits(rr) || !finite_bits(tt[2])) status = CG_ENAN;
                else if (bnorm == 0.0) { status = CG_OK; zero_b = 1; rr = 0.0; }
                else if (sqrt(rr) <= P.tol * bnorm) status = CG_OK;
                else if (o == P.max_outer || inner_total >= P.maxit) status = CG_ENOCONV;
                else if (!(tt[2] > 0.0)) status = CG_EBREAKDOWN;
                else go = 1;
                bcast[0] = tt[2];                       // rho of the inner start
                bcast[1] = P.inner_tol * sqrt(tt[0]);   // inner target on ||r32||
                ctl[kCtlRun] = go;
                ctl[kCtlZeroB] = zero_b;
            }
            __syncthreads();
            if (ctl[kCtlZeroB])
                for (int t = t0; t < t1; t += kW)
                    if (t * 32 + lane < P.n) P.x[t * 32 + lane] = 0.0;
            if (!ctl[kCtlRun]) break;
            rho = bcast[0];  // only thread 0 uses rho
        }

        // ---- inner CG in FP32 on A_lo d = r (two barriers per iteration)
        float beta = 0.0f;
        for (int k = 1;; ++k) {
            // q = A_lo z + beta q (= A_lo p), p = z + beta p; p . q
            float pq = 0.0f;
            for (int t = t0; t < t1; t += kW) {
                const float s = sell_slice_sum_lo<VT>(M, vlo, t, P.p32);
                const int row = t * 32 + lane;
                if (row < P.n) {
                    const float zi = P.p32[row];
                    const float qi = fmaf(beta, P.q32[row], fmaf(__ldg(P.diag_lo + row), zi, s));
                    const float pi = fmaf(beta, P.pd32[row], zi);
                    P.q32[row] = qi;
                    P.pd32[row] = pi;
                    pq = fmaf(pi, qi, pq);
                }
            }
            double v1[1] = {(double)pq};
            block_sum_1k<1>(v1, red, quarter);
            publish_partials<1>(P, set, v1);
            if (!grid_barrier<false>(P, epoch, S)) goto out;
            double sg[1];
            grid_totals_1k<1>(P, set, sg, quarter);
            set ^= 1;
            if (tid == 0) {
                int go = 1;
                if (!finite_bits(sg[0]) || !(sg[0] > 0.0)) go = 0;  // inner breakdown: keep d
                bcast[2] = go ? rho / sg[0] : 0.0;
                ctl[kCtlRun] = go;
                if (!go && k == 1) status = finite_bits(sg[0]) ? CG_EBREAKDOWN : CG_ENAN;
            }
            __syncthreads();
            if (!ctl[kCtlRun]) break;
            const float alpha = (float)bcast[2];
            // d += alpha p, r -= alpha q, z = M r (published); r.r, r.z
            float prr = 0.0f, prz = 0.0f;
            for (int t = t0; t < t1; t += kW) {
                const int row = t * 32 + lane;
                if (row < P.n) {
                    P.d32[row] = fmaf(alpha, P.pd32[row], P.d32[row]);
                    const float ri = fmaf(-alpha, P.q32[row], P.r32[row]);
                    P.r32[row] = ri;
                    prr = fmaf(ri, ri, prr);
                    float zi = ri;
                    if (P.precond) {
                        zi = __ldg(P.dinv32 + row) * ri;
                        prz = fmaf(ri, zi, prz);
                    }
                    P.p32[row] = zi;
                }
            }
            double v2[2] = {(double)prr, (double)(P.precond ? prz : prr)};
            block_sum_1k<2>(v2, red, quarter);
            publish_partials<2>(P, set, v2);
            if (!grid_barrier<false>(P, epoch, S)) goto out;
            double t2[2];
            grid_totals_1k<2>(P, set, t2, quarter);
            set ^= 1;
            if (tid == 0) {
                ++inner_total;
                int go = 0;
                const double rin = t2[0], rho_new = t2[1];
                if (!finite_bits(rin) || !finite_bits(rho_new) || !(rho_new > 0.0)) go = 0;
                else if (sqrt(rin) <= bcast[1]) go = 0;                 // inner target met
                else if (k >= P.max_inner || inner_total >= P.maxit) go = 0;
                else go = 1;
                if (go) {
                    bcast[3] = rho_new / rho;
                    rho = rho_new;
                }
                ctl[kCtlRun] = go;
            }
            __syncthreads();
            if (!ctl[kCtlRun]) break;
            beta = (float)bcast[3];
        }
        // ---- x += d in FP64
        for (int t = t0; t < t1; t += kW)
            if (t * 32 + lane < P.n) P.x[t * 32 + lane] += (double)P.d32[t * 32 + lane];
        if (tid == 0) outer = o + 1;
        if (!grid_barrier<false>(P, epoch, S)) goto out;
    }

    if (blockIdx.x == 0 && tid == 0) {
        P.st->iters = inner_total;
        P.st->outer = outer;
        P.st->rr = rr;
        P.st->bb = bb;
        P.st->true_rr = rr;  // the outer residual is the true FP64 residual
        atomicCAS(&P.st->status, 0, status);
    }
out:
    return;
}

// y = A x in the SELL-32 layout (stand-alone SpMV).
__global__ void __launch_bounds__(kSellThreads) sell_spmv_kernel(SellMatrix M, const double *x, double *y) {
    EpiStore epi{y};
    sell_rows(M, x, epi);
}

// ------------------------------------------ the inner SpMV on its own
// y = A_lo x with the low-precision inner matrix, through the very device
// routines the refinement kernels run in their inner CG (the staged tiles of
// cg_ir_kernel, or the SELL-32 slices of cg_irsell_kernel with the same
// CTA/warp/slice mapping), so that the inner product can be checked entry by
// entry.  x is the handle's padded inner vector p32 (the window source);
// y_i = fmaf(diag_lo_i, x_i, off-diagonal sum), as in the inner iteration.
struct EpiLoStore {
    float *y;
    const float *x;
    const float *diag;
    __device__ __forceinline__ void row(int i, float s, int) { y[i] = fmaf(diag[i], x[i], s); }
};

template <class VT>
__global__ void __launch_bounds__(kThreads, 1) lo_spmv_tiles_kernel(Params P, float *y) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Smem S = carve_smem(smem_raw);
    init_pipeline(S);
    Pipe pipe;
    const VT *vlo = nullptr;
    if constexpr (sizeof(VT) == 4) vlo = reinterpret_cast<const VT *>(P.vals32);
    else vlo = reinterpret_cast<const VT *>(P.vals16);
    EpiLoStore epi{y, P.p32, P.diag_lo};
    spmv_tiles<0, VT, float, float>(P, S, pipe, vlo, P.p32, epi, true);
    drain<float, float>(P, S, pipe, P.p32);
}

template <class VT>
__global__ void __launch_bounds__(kSellSolveThreads, 1)
    lo_spmv_sell_kernel(Params P, SellMatrix M, const VT *__restrict__ vlo, const int32_t *__restrict__ cut,
                        float *y) {
    constexpr int kW = kSellSolveThreads / 32;
    const int lane = threadIdx.x & 31;
    const int t0 = cut[blockIdx.x] + (threadIdx.x >> 5), t1 = cut[blockIdx.x + 1];
    for (int t = t0; t < t1; t += kW) {
        const float s = sell_slice_sum_lo<VT>(M, vlo, t, P.p32);
        const int row = t * 32 + lane;
        if (row < P.n) y[row] = fmaf(__ldg(P.diag_lo + row), P.p32[row], s);
    }
}

// ---------------------------------------------- FP64 throughput probe
// The FP64 roofline's denominator, measured: every thread runs 8 independent
// FMA chains (enough to cover the dependent-FMA latency with 16 warps per
// SM sub-partition), 2 flops per FMA.  The result is stored only if it takes
// an impossible value, so the chains stay live and nothing is written.
__device__ double g_fp64_probe_sink;

__global__ void __launch_bounds__(512) fp64_fma_probe_kernel(int iters, double seed) {
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = seed + 1e-9 * (double)(threadIdx.x + 64 * j);
    const double m = 0.9999999999, c = 1e-12;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fma(a[j], m, c);
    }
    const double s = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    if (s == -12345.0) g_fp64_probe_sink = s;
}

constexpr int kRptChoices[] = {0, 1, 2, 4};
SolveKernel solve_kernel_for(int rpt) {
    switch (rpt) {
        case 1: return cg_solve_kernel<1>;
        case 2: return cg_solve_kernel<2>;
        case 4: return cg_solve_kernel<4>;
        default: return cg_solve_kernel<0>;
    }
}

}  // namespace

// =================================================================== host

namespace {

void free_handle(cg_handle *h) {
    if (!h) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    learn_free(h);
    for (void *p : h->allocs) cudaFree(p);
    if (h->st_host) cudaFreeHost(h->st_host);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    cudaSetDevice(prev);
    delete h;
}

}  // namespace

Params gbcg::base_params(const cg_handle *h) {
    Params P{};
    P.n = h->n;
    P.rowptr = h->rowptr;
    P.colidx = h->colidx;
    P.vals = h->vals;
    P.tiles = h->tiles;
    P.vals32 = h->vals32;
    P.vals16 = reinterpret_cast<const __nv_bfloat16 *>(h->vals16);
    P.diag_lo = h->diag_lo;
    P.dinv32 = h->dinv32;
    P.r32 = h->r32;
    P.z32 = h->z32;
    P.p32 = h->p32;
    P.q32 = h->q32;
    P.pd32 = h->pd32;
    P.d32 = h->d32;
    P.inner_tol = h->opts.inner_tol;
    P.max_outer = h->opts.max_outer;
    P.max_inner = h->opts.max_inner > 0 ? h->opts.max_inner : h->n;
    P.lcol = h->lcol;
    P.segs = h->segs;
    P.cta_tile = h->cta_tile;
    P.cta_row = h->cta_row;
    P.dinv = h->dinv;
    P.r = h->r;
    P.z = h->z;
    P.p0 = h->p0;
    P.pd = h->pd;
    P.q = h->q;
    P.partials = h->partials;
    P.bar = h->bar;
    P.st = h->st;
    P.precond = h->opts.precond;
    P.true_res = h->opts.true_residual;
    P.phantom = h->opts.debug_phantom_arrivals;
    double w = h->opts.wait_limit_s;
    P.wait_ns = (unsigned long long)(w * 1e9);
    P.evict_first = h->evict_first;
    return P;
}

namespace {

// Enqueues one solve on the handle's stream (no synchronization).
int enqueue_solve(cg_handle *h, const double *b, double *x, double tol, int32_t maxit, int precond) {
    Params P = base_params(h);
    P.b = b;
    P.x = x;
    P.tol = tol;
    P.maxit = maxit;
    P.precond = precond;
    if (!precond) P.z = h->r;
    cudaError_t e = cudaMemsetAsync(h->bar, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->st, 0, sizeof(DevStatus), h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev0, h->stream);
    if (e == cudaSuccess) {
        if ((h->sell_solve || h->sell_mem) && h->opts.inner_values == CG_VALUES_FP64) {
            SellMatrix M = sell_of(h);
            const int32_t *cut = h->sell_cut;
            void *args[] = {&P, &M, &cut};
            const void *kern =
                h->sell_solve ? (precond ? (const void *)cg_sell_kernel<true> : (const void *)cg_sell_kernel<false>)
                              : (precond ? (const void *)cg_sellmem_kernel<true>
                                         : (const void *)cg_sellmem_kernel<false>);
            e = cudaLaunchCooperativeKernel(kern, dim3(h->ctas), dim3(kSellSolveThreads), args, 0, h->stream);
        } else if (h->sell_lo && h->opts.inner_values != CG_VALUES_FP64) {
            SellMatrix M = sell_of(h);
            const int32_t *cut = h->sell_cut;
            const void *vlo = h->sell_lo;
            void *args[] = {&P, &M, &vlo, &cut};
            const void *kern = h->opts.inner_values == CG_VALUES_FP32 ? (const void *)cg_irsell_kernel<float>
                                                                       : (const void *)cg_irsell_kernel<__nv_bfloat16>;
            e = cudaLaunchCooperativeKernel(kern, dim3(h->ctas), dim3(kSellSolveThreads), args, 0, h->stream);
        } else {
            void *args[] = {&P};
            const void *kern = (const void *)h->kernel;
            if (h->opts.inner_values == CG_VALUES_FP32) kern = (const void *)cg_ir_kernel<float>;
            if (h->opts.inner_values == CG_VALUES_BF16) kern = (const void *)cg_ir_kernel<__nv_bfloat16>;
            e = cudaLaunchCooperativeKernel(kern, dim3(h->ctas), dim3(kThreads),
                                            args, (size_t)kSmemBytes, h->stream);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->ev1, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->st_host, h->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream);
    return e == cudaSuccess ? CG_OK : CG_ECUDA;
}

int finish_solve(cg_handle *h, cg_info *info) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return CG_ECUDA;
    const DevStatus &s = *h->st_host;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    const double bnorm = std::sqrt(s.bb);
    cg_info out{};
    out.iters = s.iters;
    out.status = s.status;
    out.relres = bnorm > 0.0 ? std::sqrt(s.rr) / bnorm : 0.0;
    out.relres_true = s.true_rr < 0.0 ? -1.0 : (bnorm > 0.0 ? std::sqrt(s.true_rr) / bnorm : 0.0);
    out.kernel_ms = ms;
    out.launches = 1;
    out.outer = s.outer;
    out.reverted_at = -1;
    if (info) *info = out;
    return s.status;
}

int check_solve_args(const cg_handle *h, const double *b, const double *x, double tol) {
    if (!h) return CG_EINVAL;
    if (!(tol >= 0.0) || !std::isfinite(tol)) return CG_EINVAL;
    if (h->n > 0 && (!b || !x || b == x)) return CG_EINVAL;
    return CG_OK;
}

void empty_info(cg_info *info) {
    if (info) {
        *info = cg_info{};
        info->relres_true = 0.0;
        info->reverted_at = -1;
    }
}

}  // namespace

int gbcg::enqueue_fp64_solve(cg_handle *h, const double *b, double *x, double tol, int32_t maxit,
                             int precond) {
    return enqueue_solve(h, b, x, tol, maxit, precond);
}

int gbcg::enqueue_spmv(cg_handle *h, const double *x, double *y) {
    sell_spmv_kernel<<<h->sell_grid, kSellThreads, 0, h->stream>>>(sell_of(h), x, y);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ECUDA;
}

extern "C" {

int cg_version(void) { return 10000; }

int cg_opts_default(cg_opts *opts) {
    if (!opts) return CG_EINVAL;
    *opts = cg_opts{};
    opts->precond = CG_PRECOND_NONE;
    opts->true_residual = 1;
    opts->wait_limit_s = 5.0;
    opts->grid_ctas = 0;
    opts->debug_phantom_arrivals = 0;
    opts->vectors_in_memory = 0;
    opts->inner_values = CG_VALUES_FP64;
    opts->inner_tol = 0.0;
    opts->max_outer = 50;
    opts->max_inner = 0;
    return CG_OK;
}

const char *cg_strerror(int code) {
    switch (code) {
        case CG_OK: return "ok";
        case CG_EINVAL: return "invalid argument or malformed CSR matrix";
        case CG_ENOMEM: return "out of memory";
        case CG_ECUDA: return "CUDA runtime error";
        case CG_ENOCONV: return "maximum iterations reached before the tolerance";
        case CG_EBREAKDOWN: return "breakdown: matrix or preconditioner not positive definite";
        case CG_ENAN: return "NaN or infinity in a reduction";
        case CG_ETIMEOUT: return "bounded device wait timed out";
        default: return "unknown status";
    }
}

int cg_create(const cg_csr *A, const cg_opts *opts_in, void *stream, cg_handle **out) {
    NvtxRange nvtx("gbcg.create");
    if (!out) return CG_EINVAL;
    *out = nullptr;
    if (!A) return CG_EINVAL;
    cg_opts opts;
    if (opts_in) {
        opts = *opts_in;
    } else {
        cg_opts_default(&opts);
    }
    if (opts.precond != CG_PRECOND_NONE && opts.precond != CG_PRECOND_JACOBI && opts.precond != CG_PRECOND_LEARNED)
        return CG_EINVAL;
    if (opts.precond == CG_PRECOND_LEARNED && opts.inner_values != CG_VALUES_FP64) return CG_EINVAL;
    if (!(opts.wait_limit_s > 0.0) || !std::isfinite(opts.wait_limit_s) || opts.wait_limit_s > 3600.0)
        return CG_EINVAL;
    if (opts.grid_ctas < 0 || opts.debug_phantom_arrivals < 0 || opts.debug_phantom_arrivals > 1024)
        return CG_EINVAL;
    if (opts.vectors_in_memory != 0 && opts.vectors_in_memory != 1) return CG_EINVAL;
    if (opts.inner_values != CG_VALUES_FP64 && opts.inner_values != CG_VALUES_FP32 &&
        opts.inner_values != CG_VALUES_BF16)
        return CG_EINVAL;
    if (opts.inner_tol == 0.0) opts.inner_tol = opts.inner_values == CG_VALUES_BF16 ? 1e-2 : 1e-3;
    if (!(opts.inner_tol > 0.0 && opts.inner_tol < 1.0) || opts.max_outer < 1 || opts.max_inner < 0)
        return CG_EINVAL;
    const int32_t n = A->n;
    const int64_t nnz = A->nnz;
    if (n < 0 || nnz < 0 || nnz > (int64_t)INT32_MAX - 64) return CG_EINVAL;
    if (A->mem != CG_MEM_HOST && A->mem != CG_MEM_DEVICE) return CG_EINVAL;
    if (!A->rowptr) return CG_EINVAL;
    if (nnz > 0 && (!A->colidx || !A->vals)) return CG_EINVAL;

    // ---- host copies of the matrix for validation and planning (host-side
    // matrices are validated before any CUDA call)
    std::vector<int32_t> rowptr(n + 1), colidx(nnz);
    std::vector<double> vals(nnz);
    if (A->mem == CG_MEM_DEVICE) {
        if (cudaMemcpy(rowptr.data(), A->rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return CG_EINVAL;
        if (nnz > 0 &&
            (cudaMemcpy(colidx.data(), A->colidx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost) !=
                 cudaSuccess ||
             cudaMemcpy(vals.data(), A->vals, sizeof(double) * nnz, cudaMemcpyDeviceToHost) !=
                 cudaSuccess))
            return CG_EINVAL;
    } else {
        std::memcpy(rowptr.data(), A->rowptr, sizeof(int32_t) * (n + 1));
        if (nnz > 0) {
            std::memcpy(colidx.data(), A->colidx, sizeof(int32_t) * nnz);
            std::memcpy(vals.data(), A->vals, sizeof(double) * nnz);
        }
    }
    if (rowptr[0] != 0 || (int64_t)rowptr[n] != nnz) return CG_EINVAL;
    for (int32_t i = 0; i < n; ++i)
        if (rowptr[i + 1] < rowptr[i]) return CG_EINVAL;
    for (int64_t k = 0; k < nnz; ++k)
        if (colidx[k] < 0 || colidx[k] >= n) return CG_EINVAL;

    std::vector<double> dinv;
    if (opts.precond != CG_PRECOND_NONE) {
        dinv.resize(n);
        for (int32_t i = 0; i < n; ++i) {
            double d = 0.0;
            for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
                if (colidx[k] == i) d += vals[k];
            if (!(d > 0.0) || !std::isfinite(d)) return CG_EINVAL;
            dinv[i] = 1.0 / d;
        }
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CG_ECUDA;

    cg_handle *h = new (std::nothrow) cg_handle();
    if (!h) return CG_ENOMEM;
    h->device = dev;
    h->stream = static_cast<cudaStream_t>(stream);
    h->opts = opts;
    h->n = n;
    h->nnz = nnz;

    int rc = CG_OK;
    auto fail = [&](int code) {
        free_handle(h);
        return code;
    };

    // ---- plan: tiles, CTAs
    int max_tile = 0;
    std::vector<int32_t> tiles = n > 0 ? plan_tiles(n, rowptr, &max_tile) : std::vector<int32_t>{0};
    h->ntiles = (int)tiles.size() - 1;
    h->max_tile_nnz = max_tile;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return fail(CG_ECUDA);
    for (int rpt : kRptChoices) {
        if (cudaFuncSetAttribute((const void *)solve_kernel_for(rpt),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess)
            return fail(CG_ECUDA);
    }
    if (cudaFuncSetAttribute((const void *)sell_spmv_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxL1) != cudaSuccess ||
        cudaFuncSetAttribute((const void *)cg_ir_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemBytes) != cudaSuccess ||
        cudaFuncSetAttribute((const void *)cg_ir_kernel<__nv_bfloat16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess ||
        cudaFuncSetAttribute((const void *)lo_spmv_tiles_kernel<float>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess ||
        cudaFuncSetAttribute((const void *)lo_spmv_tiles_kernel<__nv_bfloat16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess)
        return fail(CG_ECUDA);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_kernel_for(4), kThreads, kSmemBytes) !=
            cudaSuccess ||
        per_sm < 1)
        return fail(CG_ECUDA);
    const int max_ctas = sms * per_sm;
    int ctas = opts.grid_ctas > 0 ? std::min(opts.grid_ctas, max_ctas) : sms;
    ctas = std::max(1, std::min(ctas, std::max(1, h->ntiles)));
    h->ctas = ctas;
    std::vector<int32_t> cut = split_tiles(tiles, rowptr, ctas);
    // rows per thread: warp 0 of the CTA with the most tiles owns the most
    int max_tiles = 0;
    for (int c = 0; c < ctas; ++c) max_tiles = std::max(max_tiles, cut[c + 1] - cut[c]);
    const int per_warp = (max_tiles + kWarps - 1) / kWarps;
    h->rpt = 0;
    if (!opts.vectors_in_memory) {
        for (int rpt : kRptChoices)
            if (rpt > 0 && per_warp <= rpt) {
                h->rpt = rpt;
                break;
            }
    }
    h->kernel = solve_kernel_for(h->rpt);
    TilePlan tp = plan_windows(n, rowptr, colidx, tiles);
    h->window_tiles = tp.windowed;
    std::vector<int32_t> cta_row(ctas + 1);
    for (int c = 0; c <= ctas; ++c) cta_row[c] = tiles[cut[c]];

    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    const double matrix_bytes = 12.0 * (double)nnz + 4.0 * (n + 1);
    const double vector_bytes = 64.0 * (double)n;
    h->evict_first = (matrix_bytes + vector_bytes > 0.6 * (double)l2) ? 1 : 0;

    // ---- device memory
    const size_t pad = 16;
    if ((rc = dev_alloc(h, &h->rowptr, (size_t)n + 1 + pad)) ||
        (rc = dev_alloc(h, &h->colidx, (size_t)nnz + pad)) ||
        (rc = dev_alloc(h, &h->vals, (size_t)nnz + pad)) ||
        (rc = dev_alloc(h, &h->tiles, tp.desc.size())) ||
        (rc = dev_alloc(h, &h->segs, tp.segs.size())) ||
        (rc = dev_alloc(h, &h->lcol, tp.lcol.size())) ||
        (rc = dev_alloc(h, &h->cta_tile, cut.size())) ||
        (rc = dev_alloc(h, &h->cta_row, cta_row.size())) ||
        (rc = dev_alloc(h, &h->r, (size_t)n)) ||
        (rc = dev_alloc(h, &h->p0, (size_t)n + pad)) ||
        (rc = dev_alloc(h, &h->q, (size_t)n)) ||
        (rc = dev_alloc(h, &h->pd, (size_t)n)) ||
        (rc = dev_alloc(h, &h->b_dev, (size_t)n)) ||
        (rc = dev_alloc(h, &h->x_dev, (size_t)n + pad)) ||
        (rc = dev_alloc(h, &h->partials, (size_t)2 * ctas * kRedSlots)) ||
        (rc = dev_alloc(h, &h->bar, 64)) ||
        (rc = dev_alloc(h, &h->st, 1)))
        return fail(rc);
    if (opts.precond != CG_PRECOND_NONE) {
        if ((rc = dev_alloc(h, &h->z, (size_t)n)) || (rc = dev_alloc(h, &h->dinv, (size_t)n))) return fail(rc);
    } else {
        h->z = h->r;
    }
    InnerMatrix inner;
    const bool mixed = opts.inner_values != CG_VALUES_FP64;
    if (mixed) {
        inner = build_inner(n, rowptr, colidx, vals, opts.inner_values == CG_VALUES_FP32 ? 1 : 2);
        if (opts.precond == CG_PRECOND_JACOBI)
            for (int32_t i = 0; i < n; ++i)
                if (!(inner.diag[i] > 0.0f) || !std::isfinite(inner.diag[i])) return fail(CG_EINVAL);
        if (opts.inner_values == CG_VALUES_FP32) {
            if ((rc = dev_alloc(h, &h->vals32, (size_t)nnz + pad))) return fail(rc);
        } else {
            if ((rc = dev_alloc(h, &h->vals16, (size_t)nnz + 2 * pad))) return fail(rc);
        }
        if ((rc = dev_alloc(h, &h->diag_lo, (size_t)n)) || (rc = dev_alloc(h, &h->r32, (size_t)n)) ||
            (rc = dev_alloc(h, &h->pd32, (size_t)n)) ||
            (rc = dev_alloc(h, &h->p32, (size_t)n + pad)) || (rc = dev_alloc(h, &h->q32, (size_t)n)) ||
            (rc = dev_alloc(h, &h->d32, (size_t)n)))
            return fail(rc);
        if (opts.precond == CG_PRECOND_JACOBI) {
            if ((rc = dev_alloc(h, &h->z32, (size_t)n)) || (rc = dev_alloc(h, &h->dinv32, (size_t)n)))
                return fail(rc);
        } else {
            h->z32 = h->r32;
        }
    }
    {   // SELL-32 copy for the stand-alone SpMV and the slice solve kernel
        SellHost sh = build_sell(n, rowptr, colidx, vals);
        h->sell_slices = (n + 31) / 32;
        h->sell_grid = std::max(1, std::min(sms * kSellBlocksPerSm, (h->sell_slices + 7) / 8));
        // the slice kernel: every warp of the h->ctas CTAs owns at most one slice
        const std::vector<int32_t> cut =
            opts.vectors_in_memory || n == 0 ? std::vector<int32_t>{}
                                             : split_slices(sh.ptr, ctas, kSliceMaxPerCta, kSliceVecCost);
        h->sell_solve = 0;
        if (!cut.empty()) {
            int occ_plain = 0, occ_pre = 0;
            const bool ok =
                cudaFuncSetAttribute((const void *)cg_sell_kernel<false>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxL1) == cudaSuccess &&
                cudaFuncSetAttribute((const void *)cg_sell_kernel<true>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxL1) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_plain, cg_sell_kernel<false>,
                                                              kSellSolveThreads, 0) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_pre, cg_sell_kernel<true>,
                                                              kSellSolveThreads, 0) == cudaSuccess;
            if (!ok) return fail(CG_ECUDA);
            if (occ_plain >= 1 && occ_pre >= 1) {
                // each row's entries in the CTA's own rows first (read while the
                // grid barrier that publishes z completes)
                sh = build_sell(n, rowptr, colidx, vals, &cut);
                if ((rc = dev_alloc(h, &h->sell_cut, cut.size())) ||
                    (rc = dev_alloc(h, &h->sell_split, sh.split.size())))
                    return fail(rc);
                if (cudaMemcpy(h->sell_cut, cut.data(), sizeof(int32_t) * cut.size(), cudaMemcpyHostToDevice) !=
                        cudaSuccess ||
                    cudaMemcpy(h->sell_split, sh.split.data(), sizeof(int32_t) * sh.split.size(),
                               cudaMemcpyHostToDevice) != cudaSuccess)
                    return fail(CG_ECUDA);
                h->sell_solve = 1;
            }
        }
        // larger systems (no register rows in the tiled kernel): the SELL-32
        // kernel with the vectors in memory, slices in contiguous ranges per CTA
        if (!h->sell_solve && !opts.vectors_in_memory && h->rpt == 0 && n > 0) {
            const std::vector<int32_t> mcut = split_slices(sh.ptr, ctas, h->sell_slices, kSliceVecCost);
            int occ_plain = 0, occ_pre = 0;
            const bool ok =
                !mcut.empty() &&
                cudaFuncSetAttribute((const void *)cg_sellmem_kernel<false>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxL1) == cudaSuccess &&
                cudaFuncSetAttribute((const void *)cg_sellmem_kernel<true>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxL1) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_plain, cg_sellmem_kernel<false>,
                                                              kSellSolveThreads, 0) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_pre, cg_sellmem_kernel<true>,
                                                              kSellSolveThreads, 0) == cudaSuccess;
            if (ok && occ_plain >= 1 && occ_pre >= 1) {
                if ((rc = dev_alloc(h, &h->sell_cut, mcut.size()))) return fail(rc);
                if (cudaMemcpy(h->sell_cut, mcut.data(), sizeof(int32_t) * mcut.size(), cudaMemcpyHostToDevice) !=
                    cudaSuccess)
                    return fail(CG_ECUDA);
                h->sell_mem = 1;
            }
        }
        // refinement on the SELL copies, for the systems of the slice kernel:
        // the low-precision off-diagonals in the same layout (the builder on
        // the low values widened to double: FP32 and BF16 values are exact in
        // double, diagonal slots stay 0).  Larger systems keep the tiled
        // refinement kernel, whose inner iteration hides more memory latency
        // (measured at 100^3: 59 against 77 us per FP32 inner iteration).
        if (mixed && h->sell_solve) {
            int occ32 = 0, occ16 = 0;
            const bool ok =
                cudaFuncSetAttribute((const void *)cg_irsell_kernel<float>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxL1) == cudaSuccess &&
                cudaFuncSetAttribute((const void *)cg_irsell_kernel<__nv_bfloat16>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxL1) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ32, cg_irsell_kernel<float>,
                                                              kSellSolveThreads, 0) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ16, cg_irsell_kernel<__nv_bfloat16>,
                                                              kSellSolveThreads, 0) == cudaSuccess;
            if (ok && occ32 >= 1 && occ16 >= 1) {
                const bool fp32 = opts.inner_values == CG_VALUES_FP32;
                std::vector<double> lo((size_t)nnz);
                for (size_t k = 0; k < (size_t)nnz; ++k)
                    lo[k] = fp32 ? (double)inner.vals32[k] : bf16_to_double(inner.vals16[k]);
                const SellHost sl = build_sell(n, rowptr, colidx, lo, &cut);
                const size_t tl = sl.vals.size();
                cudaError_t el = cudaSuccess;
                if (fp32) {
                    std::vector<float> v32(tl);
                    for (size_t k = 0; k < tl; ++k) v32[k] = (float)sl.vals[k];
                    float *d = nullptr;
                    if ((rc = dev_alloc(h, &d, tl))) return fail(rc);
                    if (tl) el = cudaMemcpy(d, v32.data(), sizeof(float) * tl, cudaMemcpyHostToDevice);
                    h->sell_lo = d;
                } else {
                    std::vector<uint16_t> v16(tl);
                    for (size_t k = 0; k < tl; ++k) v16[k] = bf16_bits_rne(sl.vals[k]);
                    uint16_t *d = nullptr;
                    if ((rc = dev_alloc(h, &d, tl))) return fail(rc);
                    if (tl) el = cudaMemcpy(d, v16.data(), sizeof(uint16_t) * tl, cudaMemcpyHostToDevice);
                    h->sell_lo = d;
                }
                if (el != cudaSuccess) return fail(cuda_fail(el));
            }
        }
        const size_t tot = sh.vals.size();
        if ((rc = dev_alloc(h, &h->sell_ptr, sh.ptr.size())) || (rc = dev_alloc(h, &h->sell_vals, tot)))
            return fail(rc);
        if (sh.rel16) rc = dev_alloc(h, &h->sell_c16, tot);
        else rc = dev_alloc(h, &h->sell_c32, tot);
        if (rc) return fail(rc);
        cudaError_t es = cudaMemcpy(h->sell_ptr, sh.ptr.data(), sizeof(long long) * sh.ptr.size(),
                                    cudaMemcpyHostToDevice);
        if (es == cudaSuccess && tot)
            es = cudaMemcpy(h->sell_vals, sh.vals.data(), sizeof(double) * tot, cudaMemcpyHostToDevice);
        if (es == cudaSuccess && tot)
            es = sh.rel16 ? cudaMemcpy(h->sell_c16, sh.cols16.data(), 2 * tot, cudaMemcpyHostToDevice)
                          : cudaMemcpy(h->sell_c32, sh.cols32.data(), 4 * tot, cudaMemcpyHostToDevice);
        if (es != cudaSuccess) return fail(cuda_fail(es));
    }
    if (cudaMallocHost(&h->st_host, sizeof(DevStatus)) != cudaSuccess) return fail(CG_ENOMEM);
    if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess)
        return fail(CG_ECUDA);

    cudaError_t e = cudaMemset(h->rowptr, 0, sizeof(int32_t) * (n + 1 + pad));
    if (e == cudaSuccess)
        e = cudaMemcpy(h->rowptr, rowptr.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->colidx, 0, sizeof(int32_t) * (nnz + pad));
    if (e == cudaSuccess) e = cudaMemset(h->vals, 0, sizeof(double) * (nnz + pad));
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpy(h->colidx, colidx.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpy(h->vals, vals.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->tiles, tp.desc.data(), sizeof(I4) * tp.desc.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->segs, tp.segs.data(), sizeof(I4) * tp.segs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->lcol, tp.lcol.data(), sizeof(uint16_t) * tp.lcol.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->p0, 0, sizeof(double) * (n + pad));
    if (e == cudaSuccess) e = cudaMemset(h->x_dev, 0, sizeof(double) * (n + pad));
    if (e == cudaSuccess)
        e = cudaMemcpy(h->cta_tile, cut.data(), sizeof(int32_t) * cut.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->cta_row, cta_row.data(), sizeof(int32_t) * cta_row.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && opts.precond != CG_PRECOND_NONE && n > 0)
        e = cudaMemcpy(h->dinv, dinv.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && mixed && n > 0) {
        if (opts.inner_values == CG_VALUES_FP32) {
            e = cudaMemset(h->vals32, 0, sizeof(float) * (nnz + pad));
            if (e == cudaSuccess && nnz > 0)
                e = cudaMemcpy(h->vals32, inner.vals32.data(), sizeof(float) * nnz, cudaMemcpyHostToDevice);
        } else {
            e = cudaMemset(h->vals16, 0, sizeof(uint16_t) * (nnz + 2 * pad));
            if (e == cudaSuccess && nnz > 0)
                e = cudaMemcpy(h->vals16, inner.vals16.data(), sizeof(uint16_t) * nnz, cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess)
            e = cudaMemcpy(h->diag_lo, inner.diag.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(h->p32, 0, sizeof(float) * (n + pad));
        if (e == cudaSuccess && opts.precond == CG_PRECOND_JACOBI) {
            std::vector<float> di(n);
            for (int32_t i = 0; i < n; ++i) di[i] = 1.0f / inner.diag[i];
            e = cudaMemcpy(h->dinv32, di.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
        }
    }
    if (e != cudaSuccess) return fail(cuda_fail(e));
    *out = h;
    return CG_OK;
}

static int solve_device(cg_handle *h, const double *b, double *x, double tol, int32_t maxit, cg_info *info) {
    NvtxRange nvtx("gbcg.solve");
    int rc = check_solve_args(h, b, x, tol);
    if (rc != CG_OK) return rc;
    if (h->n == 0) {
        empty_info(info);
        return CG_OK;
    }
    DeviceGuard g(h->device);
    if (maxit <= 0) maxit = h->n;
    if (h->opts.precond == CG_PRECOND_LEARNED) return learn_solve(h, b, x, tol, maxit, info);
    // The solve works on the handle's padded, 16-byte aligned copy of x (the
    // TMA copies of x-windows need that alignment), copied in and out on the
    // stream.
    const size_t bytes = sizeof(double) * (size_t)h->n;
    if (cudaMemcpyAsync(h->x_dev, x, bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
        return CG_ECUDA;
    if ((rc = enqueue_solve(h, b, h->x_dev, tol, maxit, h->opts.precond)) != CG_OK) return rc;
    if (cudaMemcpyAsync(x, h->x_dev, bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
        return CG_ECUDA;
    return finish_solve(h, info);
}

static int solve_host(cg_handle *h, const double *b, double *x, double tol, int32_t maxit, cg_info *info) {
    NvtxRange nvtx("gbcg.solve_host");
    int rc = check_solve_args(h, b, x, tol);
    if (rc != CG_OK) return rc;
    if (h->n == 0) {
        empty_info(info);
        return CG_OK;
    }
    DeviceGuard g(h->device);
    if (maxit <= 0) maxit = h->n;
    const size_t bytes = sizeof(double) * (size_t)h->n;
    if (cudaMemcpyAsync(h->b_dev, b, bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->x_dev, x, bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return CG_ECUDA;
    if (h->opts.precond == CG_PRECOND_LEARNED) {
        rc = learn_solve(h, h->b_dev, h->x_dev, tol, maxit, info);
        if (cudaMemcpyAsync(x, h->x_dev, bytes, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            return CG_ECUDA;
        return rc;
    }
    if ((rc = enqueue_solve(h, h->b_dev, h->x_dev, tol, maxit, h->opts.precond)) != CG_OK) return rc;
    if (cudaMemcpyAsync(x, h->x_dev, bytes, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return CG_ECUDA;
    return finish_solve(h, info);
}

// info->status is the return code whether or not the solve ran: a call that
// fails before the solve (bad arguments, a CUDA error) leaves a result with
// that status and nothing else.
static constexpr int32_t kInfoUnset = INT32_MIN;
static void settle_info(cg_info *info, int rc) {
    if (!info) return;
    if (info->status == kInfoUnset) {
        *info = cg_info{};
        info->relres_true = -1.0;
        info->reverted_at = -1;
    }
    info->status = rc;
}

int cg_solve(cg_handle *h, const double *b, double *x, double tol, int32_t maxit, cg_info *info) {
    if (info) info->status = kInfoUnset;
    const int rc = solve_device(h, b, x, tol, maxit, info);
    settle_info(info, rc);
    return rc;
}

int cg_solve_host(cg_handle *h, const double *b, double *x, double tol, int32_t maxit, cg_info *info) {
    if (info) info->status = kInfoUnset;
    const int rc = solve_host(h, b, x, tol, maxit, info);
    settle_info(info, rc);
    return rc;
}

int cg_spmv(cg_handle *h, const double *x, double *y) {
    NvtxRange nvtx("gbcg.spmv");
    if (!h) return CG_EINVAL;
    if (h->n == 0) return CG_OK;
    if (!x || !y || x == y) return CG_EINVAL;
    DeviceGuard g(h->device);
    return enqueue_spmv(h, x, y);
}

int cg_spmv_inner(cg_handle *h, const float *x, float *y) {
    NvtxRange nvtx("gbcg.spmv_inner");
    if (!h || h->opts.inner_values == CG_VALUES_FP64) return CG_EINVAL;
    if (h->n == 0) return CG_OK;
    if (!x || !y) return CG_EINVAL;
    DeviceGuard g(h->device);
    // the inner kernels gather from the handle's padded, 16-byte aligned p32
    cudaError_t e = cudaMemcpyAsync(h->p32, x, sizeof(float) * (size_t)h->n, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->st, 0, sizeof(DevStatus), h->stream);
    if (e == cudaSuccess) {
        Params P = base_params(h);
        const bool fp32 = h->opts.inner_values == CG_VALUES_FP32;
        if (h->sell_lo) {
            const SellMatrix M = sell_of(h);
            if (fp32)
                lo_spmv_sell_kernel<float><<<h->ctas, kSellSolveThreads, 0, h->stream>>>(
                    P, M, static_cast<const float *>(h->sell_lo), h->sell_cut, y);
            else
                lo_spmv_sell_kernel<__nv_bfloat16><<<h->ctas, kSellSolveThreads, 0, h->stream>>>(
                    P, M, static_cast<const __nv_bfloat16 *>(h->sell_lo), h->sell_cut, y);
        } else if (fp32) {
            lo_spmv_tiles_kernel<float><<<h->ctas, kThreads, kSmemBytes, h->stream>>>(P, y);
        } else {
            lo_spmv_tiles_kernel<__nv_bfloat16><<<h->ctas, kThreads, kSmemBytes, h->stream>>>(P, y);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->st_host, h->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return CG_ECUDA;
    return h->st_host->status;   // CG_OK, or CG_ETIMEOUT if a TMA wait ran out
}

int cg_get_plan(const cg_handle *h, cg_plan *plan) {
    if (!h || !plan) return CG_EINVAL;
    cg_plan p{};
    p.n = h->n;
    p.nnz = h->nnz;
    p.ctas = h->ctas;
    p.threads = kThreads;
    p.tiles = h->ntiles;
    p.tile_nnz = h->max_tile_nnz;
    p.stages = kWarps;  // one TMA stage per warp
    p.smem_bytes = kSmemBytes;
    p.lanes_per_row = 1;
    p.l2_evict_first = h->evict_first;
    p.reg_rows = h->rpt;
    p.window_tiles = h->window_tiles;
    p.device_bytes = h->device_bytes;
    p.slice_solve = h->sell_solve ? 1 : (h->sell_mem ? 2 : 0);
    p.inner_solve = h->sell_lo ? 1 : 0;
    *plan = p;
    return CG_OK;
}

void cg_destroy(cg_handle *h) { free_handle(h); }

int cg_bounds_faults(int64_t *count) {
    if (!count) return CG_EINVAL;
    const long long parts[] = {read_bounds_faults(), bounds_faults_batch(), bounds_faults_learn()};
    long long tot = 0;
    for (long long v : parts) {
        if (v < 0) {
            *count = -1;
            return CG_OK;
        }
        tot += v;
    }
    *count = tot;
    return CG_OK;
}

int cg_fp64_peak(void *stream, int32_t iters, double *flops, double *ms) {
    if (iters < 1 || !flops || !ms) return CG_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CG_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int blocks = sms * 4, threads = 512;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CG_ECUDA;
    fp64_fma_probe_kernel<<<blocks, threads, 0, st>>>(iters / 8 + 1, 1.0);   // warm-up
    cudaEventRecord(e0, st);
    fp64_fma_probe_kernel<<<blocks, threads, 0, st>>>(iters, 1.0);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    float t = 0.0f;
    if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return CG_ECUDA;
    *flops = 2.0 * 8.0 * (double)iters * (double)blocks * (double)threads;
    *ms = (double)t;
    return CG_OK;
}

}  // extern "C"
