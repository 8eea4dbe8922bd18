// S7: the macro Q4 problem of the monolithic scheme.
//
// Section 3, Eqs. (linSys), (linSys2): macro residual R^A = sum_b eta_b s_b grad N^A(X_b)
//   over the macro Gauss points b (Dirac basis: one RVE per point, Eq. (fluctVaria_dirac)),
//   with s_b = Pbar_b for R_macro and s_b = sigma_eff_b for the condensed right-hand side.
// Section 4.2, Eq. (solution2): [K - D L^-1 E] dq = -[R_macro - D L^-1 R_micro], i.e.
//   K = sum_b eta_b B_b^T Cbar_b B_b with the condensed RVE tangents, solved on the free
//   (non-Dirichlet) DOFs by a band Cholesky; then q += dq and dFbar_b = B_b dq.
// Kinematics: Fbar_b = sum_A q_A (x) grad N^A(X_b) (Section 2.1, F = grad x).
#include <algorithm>
#include <vector>

#include "fe2_internal.cuh"

namespace fe2 {

namespace {

__global__ void k_macro_gradients(MacroDev M, double* __restrict__ Fbar, double* __restrict__ eta_out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= M.ngp) return;
    const int e = b >> 2;
    double F[4] = {0.0, 0.0, 0.0, 0.0};
    for (int A = 0; A < 4; ++A) {
        const int n = M.conn[4 * e + A];
        for (int i = 0; i < 2; ++i)
            for (int J = 0; J < 2; ++J) F[2 * i + J] += M.q[2 * n + i] * M.grads[(b * 4 + A) * 2 + J];
    }
    for (int k = 0; k < 4; ++k) Fbar[4 * b + k] = F[k];
    if (eta_out) eta_out[b] = M.eta[b];
}

// One thread per free row (node A, comp c): row entries of K (lower part into
// the band columns) and R, accumulated in a fixed order over the node's elements.
__global__ void k_macro_assemble(MacroDev M, const double* __restrict__ stress, const double* __restrict__ Cbar,
                                 int with_K) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * M.nnode) return;
    const int i = M.dof2free[t];
    if (i < 0) return;
    const int A = t >> 1, c = t & 1;
    const int LD = M.kd + 1;
    double r = 0.0;
    for (int p = M.adj_ptr[A]; p < M.adj_ptr[A + 1]; ++p) {
        const int e = M.adj[p] >> 2, a = M.adj[p] & 3;
        for (int q = 0; q < 4; ++q) {
            const int b = 4 * e + q;
            const double* G = M.grads + (size_t)b * 8;
            const double eta = M.eta[b];
            r += eta * (stress[4 * b + 2 * c] * G[2 * a] + stress[4 * b + 2 * c + 1] * G[2 * a + 1]);
            if (!with_K) continue;
            const double* C = Cbar + (size_t)b * 16;
            // t_kL = sum_J G_aJ C[cJ][kL]
            double tk[4];
            for (int kL = 0; kL < 4; ++kL) tk[kL] = G[2 * a] * C[(2 * c) * 4 + kL] + G[2 * a + 1] * C[(2 * c + 1) * 4 + kL];
            for (int Bn = 0; Bn < 4; ++Bn) {
                const int nb = M.conn[4 * e + Bn];
                for (int k = 0; k < 2; ++k) {
                    const int j = M.dof2free[2 * nb + k];
                    if (j < 0 || j > i) continue;
                    const double v = eta * (tk[2 * k] * G[2 * Bn] + tk[2 * k + 1] * G[2 * Bn + 1]);
                    M.K[(size_t)j * LD + (i - j)] += v;
                }
            }
        }
    }
    M.R[i] = r - M.fext[t];  // internal minus external virtual work (Eq. (weakMech))
}

// Element RVEs (piecewise-constant basis): the condensed tangent couples the
// four Gauss points of an element, Cbar_e[(4g + iJ)][(4g' + kL)] (16 x 16), so
// K_AB = sum_e sum_g sum_g' eta_g B_g(A)^T Cbar_e[g][g'] B_g'(B).  R as above.
__global__ void k_macro_assemble_elem(MacroDev M, const double* __restrict__ stress, const double* __restrict__ Cbar) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * M.nnode) return;
    const int i = M.dof2free[t];
    if (i < 0) return;
    const int A = t >> 1, c = t & 1;
    const int LD = M.kd + 1;
    double r = 0.0;
    for (int p = M.adj_ptr[A]; p < M.adj_ptr[A + 1]; ++p) {
        const int e = M.adj[p] >> 2, a = M.adj[p] & 3;
        const double* Ce = Cbar + (size_t)e * 256;
        for (int g = 0; g < 4; ++g) {
            const int b = 4 * e + g;
            const double* G = M.grads + (size_t)b * 8;
            const double eta = M.eta[b];
            r += eta * (stress[4 * b + 2 * c] * G[2 * a] + stress[4 * b + 2 * c + 1] * G[2 * a + 1]);
            for (int g2 = 0; g2 < 4; ++g2) {
                const double* G2 = M.grads + (size_t)(4 * e + g2) * 8;
                // tk_kL = sum_J G_aJ Cbar_e[(g, c, J)][(g2, kL)]
                double tk[4];
                for (int kL = 0; kL < 4; ++kL)
                    tk[kL] = G[2 * a] * Ce[(4 * g + 2 * c) * 16 + 4 * g2 + kL] +
                             G[2 * a + 1] * Ce[(4 * g + 2 * c + 1) * 16 + 4 * g2 + kL];
                for (int Bn = 0; Bn < 4; ++Bn) {
                    const int nb = M.conn[4 * e + Bn];
                    for (int k = 0; k < 2; ++k) {
                        const int j = M.dof2free[2 * nb + k];
                        if (j < 0 || j > i) continue;
                        M.K[(size_t)j * LD + (i - j)] += eta * (tk[2 * k] * G2[2 * Bn] + tk[2 * k + 1] * G2[2 * Bn + 1]);
                    }
                }
            }
        }
    }
    M.R[i] = r - M.fext[t];
}

// One CTA: ||R||_2 of the free residual (deterministic tree).
__global__ void k_macro_norm(MacroDev M, double* __restrict__ out) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < M.nfree; i += blockDim.x) s += M.R[i] * M.R[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sqrt(red[0]);
}

// One CTA: in-place band Cholesky of K (FP64), then K dq_free = -R.
__global__ void __launch_bounds__(1024) k_macro_chol_solve(MacroDev M, int* __restrict__ status) {
    const int n = M.nfree, kd = M.kd, LD = kd + 1;
    double* K = M.K;
    __shared__ int bad;
    __shared__ double dj;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        double* Lj = K + (size_t)j * LD;
        if (threadIdx.x == 0) {
            double p = Lj[0];
            if (!(p > 0.0)) {
                bad = 1;
                p = 1.0;
            }
            dj = sqrt(p);
            Lj[0] = dj;
        }
        __syncthreads();
        const int m = min(kd, n - 1 - j);
        for (int r = 1 + threadIdx.x; r <= m; r += blockDim.x) Lj[r] /= dj;
        __syncthreads();
        // trailing update: column j+u (u = 1..m), rows j+u .. j+m
        {
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
            for (int u = 1 + warp; u <= m; u += nw) {
                const double lu = Lj[u];
                double* Ku = K + (size_t)(j + u) * LD;
                for (int v = u + lane; v <= m; v += 32) Ku[v - u] -= Lj[v] * lu;
            }
        }
        __syncthreads();
    }
    // forward (one warp, column sweep) then backward (one warp, dot products)
    double* y = M.R;  // overwritten: y = L^-1 (-R), then x = L^-T y
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int i = lane; i < n; i += 32) y[i] = -y[i];
        __syncwarp();
        for (int j = 0; j < n; ++j) {
            const double* Lj = K + (size_t)j * LD;
            const double yj = y[j] / Lj[0];
            __syncwarp();
            if (lane == 0) y[j] = yj;
            const int m = min(kd, n - 1 - j);
            for (int r = 1 + lane; r <= m; r += 32) y[j + r] -= Lj[r] * yj;
            __syncwarp();
        }
        for (int j = n - 1; j >= 0; --j) {
            const double* Lj = K + (size_t)j * LD;
            const int m = min(kd, n - 1 - j);
            double s = 0.0;
            for (int r = 1 + lane; r <= m; r += 32) s += Lj[r] * y[j + r];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) y[j] = (y[j] - s) / Lj[0];
            __syncwarp();
        }
    }
    if (threadIdx.x == 0 && status) *status = bad ? FE2_ERR_NOT_PD : FE2_OK;
}

// dq on all DOFs (zero on fixed ones), q += dq, dFbar_b = B_b dq.
__global__ void k_macro_apply(MacroDev M, double* __restrict__ dFbar) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 2 * M.nnode) {
        const int f = M.dof2free[t];
        const double d = f >= 0 ? M.R[f] : 0.0;
        M.dq[t] = d;
    }
}
__global__ void k_macro_apply2(MacroDev M, double* __restrict__ dFbar) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < M.ngp) {
        const int e = b >> 2;
        double F[4] = {0.0, 0.0, 0.0, 0.0};
        for (int A = 0; A < 4; ++A) {
            const int n = M.conn[4 * e + A];
            for (int i = 0; i < 2; ++i)
                for (int J = 0; J < 2; ++J) F[2 * i + J] += M.dq[2 * n + i] * M.grads[(b * 4 + A) * 2 + J];
        }
        for (int k = 0; k < 4; ++k) dFbar[4 * b + k] = F[k];
    }
}
__global__ void k_macro_apply3(MacroDev M) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 2 * M.nnode) M.q[t] += M.dq[t];
}

// Volume-averaged stress Pbar = Pint / |Omega| and ||r_m|| per RVE.
__global__ void k_rve_avg_stress(const RveDev* __restrict__ tab, const int* __restrict__ ids, int n,
                                 double* __restrict__ Pbar) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const RveDev& r = tab[ids[t]];
    const int dd = r.d * r.d;
    for (int k = 0; k < dd; ++k) Pbar[(size_t)t * dd + k] = r.Pint[k];  // |Omega| = 1
}

__global__ void k_rve_rnorm(const RveDev* __restrict__ tab, const int* __restrict__ ids, double* __restrict__ out) {
    __shared__ double red[256];
    const RveDev r = tab[ids[blockIdx.x]];
    const double* rm = r.rhs + (size_t)(r.nr - 1) * r.nm;
    double s = 0.0;
    for (int m = threadIdx.x; m < r.nm; m += blockDim.x) s += rm[m] * rm[m];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sqrt(red[0]);
}

}  // namespace

cudaError_t launch_macro_gradients(const MacroDev& M, double* Fbar, double* eta, cudaStream_t s) {
    k_macro_gradients<<<(M.ngp + 127) / 128, 128, 0, s>>>(M, Fbar, eta);
    return cudaGetLastError();
}

cudaError_t launch_macro_residual(const MacroDev& M, const double* stress, double* rnorm, cudaStream_t s) {
    k_macro_assemble<<<(2 * M.nnode + 127) / 128, 128, 0, s>>>(M, stress, nullptr, 0);
    k_macro_norm<<<1, 1024, 0, s>>>(M, rnorm);
    return cudaGetLastError();
}

cudaError_t launch_macro_solve(const MacroDev& M, const double* stress, const double* Cbar, double* dFbar,
                               double* rnorm, int* status, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(M.K, 0, sizeof(double) * (size_t)M.nfree * (M.kd + 1), s);
    if (e != cudaSuccess) return e;
    k_macro_assemble<<<(2 * M.nnode + 127) / 128, 128, 0, s>>>(M, stress, Cbar, 1);
    k_macro_norm<<<1, 1024, 0, s>>>(M, rnorm);
    k_macro_chol_solve<<<1, 1024, 0, s>>>(M, status);
    k_macro_apply<<<(2 * M.nnode + 127) / 128, 128, 0, s>>>(M, dFbar);
    k_macro_apply2<<<(M.ngp + 127) / 128, 128, 0, s>>>(M, dFbar);
    k_macro_apply3<<<(2 * M.nnode + 127) / 128, 128, 0, s>>>(M);
    return cudaGetLastError();
}

cudaError_t launch_macro_solve_elem(const MacroDev& M, const double* stress, const double* Cbar, double* dFbar,
                                    double* rnorm, int* status, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(M.K, 0, sizeof(double) * (size_t)M.nfree * (M.kd + 1), s);
    if (e != cudaSuccess) return e;
    k_macro_assemble_elem<<<(2 * M.nnode + 127) / 128, 128, 0, s>>>(M, stress, Cbar);
    k_macro_norm<<<1, 1024, 0, s>>>(M, rnorm);
    k_macro_chol_solve<<<1, 1024, 0, s>>>(M, status);
    k_macro_apply<<<(2 * M.nnode + 127) / 128, 128, 0, s>>>(M, dFbar);
    k_macro_apply2<<<(M.ngp + 127) / 128, 128, 0, s>>>(M, dFbar);
    k_macro_apply3<<<(2 * M.nnode + 127) / 128, 128, 0, s>>>(M);
    return cudaGetLastError();
}

cudaError_t launch_rve_avg_stress(const RveDev* tab, const int* ids, int n, double* Pbar, cudaStream_t s) {
    k_rve_avg_stress<<<(n + 127) / 128, 128, 0, s>>>(tab, ids, n, Pbar);
    return cudaGetLastError();
}

cudaError_t launch_rve_rnorm(const RveDev* tab, const int* ids, int n, double* out, cudaStream_t s) {
    k_rve_rnorm<<<n, 256, 0, s>>>(tab, ids, out);
    return cudaGetLastError();
}

}  // namespace fe2
