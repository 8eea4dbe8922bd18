// Element RVEs of the piecewise-constant macro basis (Section 3, Eqs.
// (constSolution1), (constSolution2)), 2D: one fluctuation w~ per macro
// element, micro residual and stiffness integrated over its nq = 4 macro Gauss
// points with weights wq (sum 1):
//   K_mm = sum_g wq_g K_mm(Fbar_g),  r_m = sum_g wq_g r_m(Fbar_g),  K_mM,g = K_mM(Fbar_g).
// rhs = [K_mM,0 | .. | K_mM,3 | r_m] (nr = 17 columns), X = K_mm^-1 rhs.  The
// condensation dw~ = -(x_r + sum_g wq_g X_M,g : dFbar_g) gives
//   Cbar[(g,iJ)][(g',kL)] = (delta_gg' K_MM,g - wq_g' K_Mm,g X_M,g')/|Omega|,
//   sigma_eff,g           = (Pint_g - K_Mm,g x_r)/|Omega|,
// on the mixed path with the FP64 residual correction of the Dirac case
// (K_Mm X -> rhs^T X + X^T R, exact up to a term quadratic in the solve error).
#include "fe2_internal.cuh"

namespace fe2 {

namespace {

constexpr int NR_E = MAX_NR;  // 17 right-hand sides
constexpr int TM = 64;                // dofs per staged tile of the Schur kernel

// FP64 residual R = rhs - K_mm X from the node-row stencil (17 columns).
__global__ void __launch_bounds__(128) k_residual2_elem(const RveDev* __restrict__ tab, const int* __restrict__ ids,
                                                        Workspace ws, const int* __restrict__ active) {
    if (active && !active[blockIdx.y]) return;
    const RveDev r = tab[ids[blockIdx.y]];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= r.nn || q == 0) return;
    const int nn = r.nn, nm = r.nm;
    double* R = (double*)(ws.base + blockIdx.y * ws.stride + ws.offR);
    double acc[2][NR_E];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int rr = 0; rr < NR_E; ++rr) acc[c][rr] = 0.0;
    for (int off = 0; off < 9; ++off) {
        const int qn = r.nbr[q * 9 + off];
        if (qn == 0) continue;
        const double k00 = r.stencil[(size_t)(off * 4 + 0) * nn + q], k01 = r.stencil[(size_t)(off * 4 + 1) * nn + q];
        const double k10 = r.stencil[(size_t)(off * 4 + 2) * nn + q], k11 = r.stencil[(size_t)(off * 4 + 3) * nn + q];
#pragma unroll
        for (int rr = 0; rr < NR_E; ++rr) {
            // the two DOFs of a node are adjacent and 16-byte aligned (nm is even)
            const double2 xv = *reinterpret_cast<const double2*>(r.X + (size_t)rr * nm + 2 * (qn - 1));
            // two chained FMAs: written as acc += a b + c d it costs a multiply, an FMA and
            // an add, and FP64 instructions set this kernel's pace
            acc[0][rr] = __fma_rn(k01, xv.y, __fma_rn(k00, xv.x, acc[0][rr]));
            acc[1][rr] = __fma_rn(k11, xv.y, __fma_rn(k10, xv.x, acc[1][rr]));
        }
    }
#pragma unroll
    for (int rr = 0; rr < NR_E; ++rr) {
        const size_t o = (size_t)rr * nm + 2 * (q - 1);
        const double2 bv = *reinterpret_cast<const double2*>(r.rhs + o);
        *reinterpret_cast<double2*>(R + o) = make_double2(bv.x - acc[0][rr], bv.y - acc[1][rr]);
    }
}

// One CTA per element RVE.  G[a][c] = sum_dof rhs_a X_c (+ X_a R_c when corrected)
// for a < 16, c < 17, accumulated over staged tiles of TM dofs; thread t owns the
// (a, c) pairs t, t + 256 (fixed order: deterministic).
__global__ void __launch_bounds__(256) k_schur2_elem(const RveDev* __restrict__ tab, const int* __restrict__ ids,
                                                     Workspace ws, int corrected, double* __restrict__ sigma,
                                                     double* __restrict__ Cbar, int* __restrict__ status,
                                                     double* __restrict__ err, const double* __restrict__ tol,
                                                     int* __restrict__ redo, int only_flagged, int final_sweep) {
    __shared__ double sB[16][TM], sX[NR_E][TM], sR[NR_E][TM];
    __shared__ double G1[16][NR_E], G2[16][NR_E];
    __shared__ double red[256][2];
    if (only_flagged && !redo[blockIdx.x]) return;
    const RveDev r = tab[ids[blockIdx.x]];
    const int nm = r.nm, tid = threadIdx.x;
    const double* __restrict__ R = (const double*)(ws.base + blockIdx.x * ws.stride + ws.offR);
    constexpr int NP = 16 * NR_E;  // 272 pairs
    double g1[2] = {0.0, 0.0}, g2[2] = {0.0, 0.0};
    for (int m0 = 0; m0 < nm; m0 += TM) {
        for (int k = tid; k < NR_E * TM; k += blockDim.x) {
            const int a = k / TM, mm = k - a * TM, m = m0 + mm;
            const bool in = m < nm;
            sX[a][mm] = in ? r.X[(size_t)a * nm + m] : 0.0;
            sR[a][mm] = (in && corrected) ? R[(size_t)a * nm + m] : 0.0;
            if (a < 16) sB[a][mm] = in ? r.rhs[(size_t)a * nm + m] : 0.0;
        }
        __syncthreads();
        for (int u = 0; u < 2; ++u) {
            const int p = tid + 256 * u;
            if (p >= NP) break;
            const int a = p / NR_E, c = p - a * NR_E;
            double s1 = 0.0, s2 = 0.0;
            for (int mm = 0; mm < TM; ++mm) {
                s1 += sB[a][mm] * sX[c][mm];
                s2 += sX[a][mm] * sR[c][mm];
            }
            g1[u] += s1;
            g2[u] += s2;
        }
        __syncthreads();
    }
    for (int u = 0; u < 2; ++u) {
        const int p = tid + 256 * u;
        if (p >= NP) break;
        const int a = p / NR_E, c = p - a * NR_E;
        G1[a][c] = g1[u];
        G2[a][c] = g2[u];
    }
    __syncthreads();
    // outputs: thread t writes Cbar entry t of the 16 x 16 block, threads < 16 sigma
    const int row = tid >> 4, col = tid & 15;  // (g, iJ) = row, (g', kL) = col
    const int g = row >> 2, g2i = col >> 2;
    const double wg2 = r.wq[g2i];
    double v = (g == g2i ? r.KMM[16 * g + 4 * (row & 3) + (col & 3)] : 0.0) - wg2 * G1[row][col];
    double corr = 0.0;
    if (corrected) {
        v -= wg2 * G2[row][col];
        corr = wg2 * G2[row][col];
    }
    Cbar[(size_t)blockIdx.x * 256 + tid] = v;  // |Omega| = 1
    int bad = !isfinite(v);
    if (tid < 16) {
        const int gq = tid >> 2;
        double sg = r.Pint[4 * gq + (tid & 3)] - G1[tid][16];
        if (corrected) sg -= G2[tid][16];
        bad |= !isfinite(sg);
        sigma[(size_t)blockIdx.x * 16 + tid] = sg;
    }
    red[tid][0] = corr * corr;
    red[tid][1] = v * v + (bad ? 1e300 : 0.0);
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (tid < o) {
            red[tid][0] += red[tid + o][0];
            red[tid][1] += red[tid + o][1];
        }
        __syncthreads();
    }
    __shared__ int s_bad;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    if (bad) s_bad = 1;
    __syncthreads();
    if (tid == 0) {
        const double e = corrected ? red[0][0] / fmax(red[0][1], 1e-300) : 0.0;
        if (err) err[blockIdx.x] = e;
        if (s_bad && status[blockIdx.x] == FE2_OK) status[blockIdx.x] = FE2_ERR_NAN;
        const bool over = corrected && !(e <= *tol);
        if (redo) redo[blockIdx.x] = (over && status[blockIdx.x] == FE2_OK) ? 1 : 0;
        if (final_sweep && over && status[blockIdx.x] == FE2_OK) status[blockIdx.x] = FE2_ERR_NO_CONV;
    }
}

// dw~ = -(x_r + sum_g wq_g X_M,g : dFbar_g), dFbar [n][nq][4].
__global__ void k_macro_update_elem(RveDev* __restrict__ tab, const int* __restrict__ ids,
                                    const double* __restrict__ dF) {
    const int id = ids[blockIdx.y];
    const RveDev r = tab[id];
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int nm = r.nm, nq = r.nq;
    if (m < nm) {
        double v = r.X[(size_t)(4 * nq) * nm + m];
        for (int g = 0; g < nq; ++g) {
            double s = 0.0;
            for (int kL = 0; kL < 4; ++kL)
                s += r.X[(size_t)(4 * g + kL) * nm + m] * dF[((size_t)blockIdx.y * nq + g) * 4 + kL];
            v += r.wq[g] * s;
        }
        r.w[m] -= v;
    }
    if (m == 0) tab[id].zero_w = 0;
}

// Pbar_g = Pint_g / |Omega| per macro Gauss point, [n][nq][4].
__global__ void k_rve_avg_stress_elem(const RveDev* __restrict__ tab, const int* __restrict__ ids, int n,
                                      double* __restrict__ Pbar) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const RveDev& r = tab[ids[t]];
    for (int k = 0; k < 4 * r.nq; ++k) Pbar[(size_t)t * 4 * r.nq + k] = r.Pint[k];
}

}  // namespace

cudaError_t launch_residual_elem(const RveDev* tab, const int* ids, int n, Workspace ws, int maxnn,
                                 const int* active, cudaStream_t s) {
    dim3 grid((maxnn + 127) / 128, n);
    k_residual2_elem<<<grid, 128, 0, s>>>(tab, ids, ws, active);
    return cudaGetLastError();
}

cudaError_t launch_schur_elem(const RveDev* tab, const int* ids, int n, Workspace ws, int corrected, double* sigma,
                              double* Cbar, int* status, double* err, const double* tol, int* redo, cudaStream_t s,
                              int refine_sweep) {
    k_schur2_elem<<<n, 256, 0, s>>>(tab, ids, ws, corrected, sigma, Cbar, status, err, tol, redo,
                                    refine_sweep == 1 || refine_sweep == 2, refine_sweep >= 2);
    return cudaGetLastError();
}

cudaError_t launch_macro_update_elem(const RveDev* tab, const int* ids, int n, const double* dF, int maxnm,
                                     cudaStream_t s) {
    dim3 grid((maxnm + 255) / 256, n);
    k_macro_update_elem<<<grid, 256, 0, s>>>(const_cast<RveDev*>(tab), ids, dF);
    return cudaGetLastError();
}

cudaError_t launch_rve_avg_stress_elem(const RveDev* tab, const int* ids, int n, double* Pbar, cudaStream_t s) {
    k_rve_avg_stress_elem<<<(n + 127) / 128, 128, 0, s>>>(tab, ids, n, Pbar);
    return cudaGetLastError();
}

}  // namespace fe2
