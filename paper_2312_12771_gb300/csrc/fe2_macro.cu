// S7: the macro Q4 (d = 2) / Hex8 (d = 3) problem of the monolithic scheme.
//
// Section 3, Eqs. (linSys), (linSys2): macro residual R^A = sum_b eta_b s_b grad N^A(X_b)
//   over the macro Gauss points b = 2^d e + q (Dirac basis: one RVE per point, Eq.
//   (fluctVaria_dirac)), with s_b = Pbar_b for R_macro and s_b = sigma_eff_b for the
//   condensed right-hand side.
// Section 4.2, Eq. (solution2): [K - D L^-1 E] dq = -[R_macro - D L^-1 R_micro], i.e.
//   K = sum_b eta_b B_b^T Cbar_b B_b with the condensed RVE tangents, solved on the free
//   (non-Dirichlet) DOFs by a blocked band Cholesky; then q += dq and dFbar_b = B_b dq.
// Kinematics: Fbar_b = sum_A q_A (x) grad N^A(X_b) (Section 2.1, F = grad x).
#include <algorithm>
#include <vector>

#include "fe2_internal.cuh"

namespace fe2 {

namespace {

constexpr int MB = 32;  // panel width of the blocked macro factorisation

template <int D>
__global__ void k_macro_gradients(MacroDev M, double* __restrict__ Fbar, double* __restrict__ eta_out) {
    constexpr int NEN = 1 << D;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= M.ngp) return;
    const int e = b / NEN;
    double F[D * D];
#pragma unroll
    for (int k = 0; k < D * D; ++k) F[k] = 0.0;
    for (int A = 0; A < NEN; ++A) {
        const int n = M.conn[NEN * e + A];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int J = 0; J < D; ++J) F[D * i + J] += M.q[D * n + i] * M.grads[((size_t)b * NEN + A) * D + J];
    }
#pragma unroll
    for (int k = 0; k < D * D; ++k) Fbar[(size_t)D * D * b + k] = F[k];
    if (eta_out) eta_out[b] = M.eta[b];
}

// One thread per free row (node A, comp c): row entries of K (lower part into
// the band columns) and R, accumulated in a fixed order over the node's elements.
template <int D>
__global__ void k_macro_assemble(MacroDev M, const double* __restrict__ stress, const double* __restrict__ Cbar,
                                 int with_K) {
    constexpr int NEN = 1 << D, DD = D * D;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= D * M.nnode) return;
    const int i = M.dof2free[t];
    if (i < 0) return;
    const int A = t / D, c = t - D * A;
    const int LD = M.kd + 1;
    double r = 0.0;
    for (int p = M.adj_ptr[A]; p < M.adj_ptr[A + 1]; ++p) {
        const int e = M.adj[p] / NEN, a = M.adj[p] - NEN * (M.adj[p] / NEN);
        for (int q = 0; q < NEN; ++q) {
            const int b = NEN * e + q;
            const double* G = M.grads + (size_t)b * NEN * D;
            const double eta = M.eta[b];
            double sr = 0.0;
#pragma unroll
            for (int J = 0; J < D; ++J) sr += stress[(size_t)DD * b + D * c + J] * G[D * a + J];
            r += eta * sr;
            if (!with_K) continue;
            const double* C = Cbar + (size_t)b * DD * DD;
            // t_kL = sum_J G_aJ C[cJ][kL]
            double tk[DD];
#pragma unroll
            for (int kL = 0; kL < DD; ++kL) {
                double v = 0.0;
#pragma unroll
                for (int J = 0; J < D; ++J) v += G[D * a + J] * C[(D * c + J) * DD + kL];
                tk[kL] = v;
            }
            for (int Bn = 0; Bn < NEN; ++Bn) {
                const int nb = M.conn[NEN * e + Bn];
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const int j = M.dof2free[D * nb + k];
                    if (j < 0 || j > i) continue;
                    double v = 0.0;
#pragma unroll
                    for (int L = 0; L < D; ++L) v += tk[D * k + L] * G[D * Bn + L];
                    M.K[(size_t)j * LD + (i - j)] += eta * v;
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

// ---------------------------------------------------------------- blocked band Cholesky
// K (n = nfree, half bandwidth kd) is stored as its lower band, column-major:
// K(i, j) = K[j (kd + 1) + i - j] for 0 <= i - j <= kd.  Panel p covers columns
// j0 .. j1 = j0 + nb - 1 (nb = min(32, n - j0)); its rows below the diagonal
// block run to rl = min(n - 1, j1 + kd).  Per panel, in stream order:
//   diag:   L11 = chol(A11)                      (one CTA)
//   trsm:   L21 = A21 L11^-T, one warp per row   (rows j1+1 .. rl)
//   update: A22 -= L21 L21^T on the trailing triangle, 32 x 32 tiles
// Entries outside the band are zero and are neither read nor written; Cholesky
// fill stays inside the band, so nothing is lost.

__device__ __forceinline__ double band_get(const MacroDev& M, int i, int j) {
    return (i - j <= M.kd) ? M.K[(size_t)j * (M.kd + 1) + (i - j)] : 0.0;
}

// Diagonal block of panel j0: one CTA of 32 x 32 threads (lane = row).
__global__ void __launch_bounds__(1024) k_mchol_diag(MacroDev M, int j0, int* __restrict__ status) {
    __shared__ double A[MB][MB + 1];
    const int n = M.nfree, nb = min(MB, n - j0);
    const int r = threadIdx.x & 31, c = threadIdx.x >> 5;
    A[r][c] = (r < nb && c < nb && r >= c) ? band_get(M, j0 + r, j0 + c) : 0.0;
    __syncthreads();
    for (int k = 0; k < nb; ++k) {
        if (threadIdx.x == 0) {
            double p = A[k][k];
            if (!(p > 0.0)) {
                *status = FE2_ERR_NOT_PD;
                p = 1.0;
            }
            A[k][k] = sqrt(p);
        }
        __syncthreads();
        if (c == k && r > k && r < nb) A[r][k] /= A[k][k];
        __syncthreads();
        if (c > k && r >= c && r < nb) A[r][c] -= A[r][k] * A[c][k];
        __syncthreads();
    }
    if (r < nb && c < nb && r >= c && r - c <= M.kd) M.K[(size_t)(j0 + c) * (M.kd + 1) + (r - c)] = A[r][c];
}

// L21 rows of panel j0: one warp per row i (lane = panel column), forward
// substitution against L11 (staged in shared memory).
__global__ void __launch_bounds__(256) k_mchol_trsm(MacroDev M, int j0) {
    __shared__ double L[MB][MB + 1];
    const int n = M.nfree, nb = min(MB, n - j0), j1 = j0 + nb - 1, rl = min(n - 1, j1 + M.kd);
    for (int t = threadIdx.x; t < MB * MB; t += blockDim.x) {
        const int r = t & 31, c = t >> 5;
        L[r][c] = (r < nb && c < nb && r >= c) ? band_get(M, j0 + r, j0 + c) : 0.0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int i = j1 + 1 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i > rl) return;
    double v = (lane < nb) ? band_get(M, i, j0 + lane) : 0.0;
    for (int k = 0; k < nb; ++k) {
        const double xk = __shfl_sync(0xffffffffu, v, k) / L[k][k];
        if (lane == k) v = xk;
        if (lane > k) v -= L[lane][k] * xk;
    }
    if (lane < nb && i - (j0 + lane) <= M.kd) M.K[(size_t)(j0 + lane) * (M.kd + 1) + (i - j0 - lane)] = v;
}

// Trailing update of panel j0: tile t -> (I, J), I >= J, of the triangle of
// rows/columns j1+1 .. rl; thread (lane = row r, s0 = warp) owns (r, s0 + 8u).
__global__ void __launch_bounds__(256) k_mchol_update(MacroDev M, int j0) {
    __shared__ double Li[MB][MB + 1];  // [panel column][tile row]
    __shared__ double Lj[MB][MB + 1];  // [tile column][panel column]
    const int n = M.nfree, nb = min(MB, n - j0), j1 = j0 + nb - 1, rl = min(n - 1, j1 + M.kd);
    int I = 0, t = blockIdx.x;
    while (t > I) {
        t -= I + 1;
        ++I;
    }
    const int J = t;
    const int i0 = j1 + 1 + MB * I, c0 = j1 + 1 + MB * J;
    for (int u = threadIdx.x; u < MB * MB; u += blockDim.x) {
        const int r = u & 31, c = u >> 5;
        const int ii = i0 + r, jj = c0 + r;
        Li[c][r] = (c < nb && ii <= rl) ? band_get(M, ii, j0 + c) : 0.0;
        Lj[r][c] = (c < nb && jj <= rl) ? band_get(M, jj, j0 + c) : 0.0;
    }
    __syncthreads();
    const int r = threadIdx.x & 31, s0 = threadIdx.x >> 5;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < nb; ++c) {
        const double li = Li[c][r];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += li * Lj[s0 + 8 * u][c];
    }
    const int i = i0 + r;
    if (i > rl) return;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int j = c0 + s0 + 8 * u;
        if (j > rl || j > i) continue;  // i - j <= kd - 1 inside the trailing triangle
        M.K[(size_t)j * (M.kd + 1) + (i - j)] -= acc[u];
    }
}

// L L^T dq = -R with the factor above, one CTA: forward then backward by panels
// (diagonal block by one warp, the band part by all threads).  dq overwrites R.
__global__ void __launch_bounds__(1024) k_mchol_solve(MacroDev M) {
    __shared__ double L[MB][MB + 1];
    __shared__ double xs[MB];
    __shared__ double part[MB];
    const int n = M.nfree, kd = M.kd;
    double* y = M.R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = -y[i];
    __syncthreads();
    const int npan = (n + MB - 1) / MB;
    for (int p = 0; p < npan; ++p) {
        const int j0 = p * MB, nb = min(MB, n - j0), j1 = j0 + nb - 1, rl = min(n - 1, j1 + kd);
        {
            const int r = threadIdx.x & 31, c = threadIdx.x >> 5;
            L[r][c] = (r < nb && c < nb && r >= c) ? band_get(M, j0 + r, j0 + c) : 0.0;
        }
        __syncthreads();
        if (warp == 0) {
            double v = lane < nb ? y[j0 + lane] : 0.0;
            for (int k = 0; k < nb; ++k) {
                const double xk = __shfl_sync(0xffffffffu, v, k) / L[k][k];
                if (lane == k) v = xk;
                if (lane > k) v -= L[lane][k] * xk;
            }
            if (lane < nb) {
                y[j0 + lane] = v;
                xs[lane] = v;
            }
        }
        __syncthreads();
        for (int i = j1 + 1 + threadIdx.x; i <= rl; i += blockDim.x) {
            double s = 0.0;
            for (int c = 0; c < nb; ++c) s += band_get(M, i, j0 + c) * xs[c];
            y[i] -= s;
        }
        __syncthreads();
    }
    for (int p = npan - 1; p >= 0; --p) {
        const int j0 = p * MB, nb = min(MB, n - j0), j1 = j0 + nb - 1, rl = min(n - 1, j1 + kd);
        {
            const int r = threadIdx.x & 31, c = threadIdx.x >> 5;
            L[r][c] = (r < nb && c < nb && r >= c) ? band_get(M, j0 + r, j0 + c) : 0.0;
        }
        // part_c = sum over the rows below the block of L(i, j0 + c) x_i (warp c)
        if (warp < nb) {
            double s = 0.0;
            for (int i = j1 + 1 + lane; i <= rl; i += 32) s += band_get(M, i, j0 + warp) * y[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) part[warp] = s;
        }
        __syncthreads();
        if (warp == 0) {
            double v = lane < nb ? y[j0 + lane] - part[lane] : 0.0;
            for (int k = nb - 1; k >= 0; --k) {
                const double xk = __shfl_sync(0xffffffffu, v, k) / L[k][k];
                if (lane == k) v = xk;
                if (lane < k) v -= L[k][lane] * xk;
            }
            if (lane < nb) y[j0 + lane] = v;
        }
        __syncthreads();
    }
}

__global__ void k_mstatus_clear(int* status) { *status = FE2_OK; }

// dq on all DOFs (zero on fixed ones), q += dq, dFbar_b = B_b dq.
__global__ void k_macro_apply(MacroDev M) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < M.d * M.nnode) {
        const int f = M.dof2free[t];
        M.dq[t] = f >= 0 ? M.R[f] : 0.0;
    }
}
template <int D>
__global__ void k_macro_apply2(MacroDev M, double* __restrict__ dFbar) {
    constexpr int NEN = 1 << D;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < M.ngp) {
        const int e = b / NEN;
        double F[D * D];
#pragma unroll
        for (int k = 0; k < D * D; ++k) F[k] = 0.0;
        for (int A = 0; A < NEN; ++A) {
            const int n = M.conn[NEN * e + A];
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int J = 0; J < D; ++J) F[D * i + J] += M.dq[D * n + i] * M.grads[((size_t)b * NEN + A) * D + J];
        }
#pragma unroll
        for (int k = 0; k < D * D; ++k) dFbar[(size_t)D * D * b + k] = F[k];
    }
}
__global__ void k_macro_apply3(MacroDev M) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < M.d * M.nnode) M.q[t] += M.dq[t];
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
    if (M.d == 3)
        k_macro_gradients<3><<<(M.ngp + 127) / 128, 128, 0, s>>>(M, Fbar, eta);
    else
        k_macro_gradients<2><<<(M.ngp + 127) / 128, 128, 0, s>>>(M, Fbar, eta);
    return cudaGetLastError();
}

static void macro_assemble(const MacroDev& M, const double* stress, const double* Cbar, int with_K, cudaStream_t s) {
    const int g = (M.d * M.nnode + 127) / 128;
    if (M.d == 3)
        k_macro_assemble<3><<<g, 128, 0, s>>>(M, stress, Cbar, with_K);
    else
        k_macro_assemble<2><<<g, 128, 0, s>>>(M, stress, Cbar, with_K);
}

cudaError_t launch_macro_residual(const MacroDev& M, const double* stress, double* rnorm, cudaStream_t s) {
    macro_assemble(M, stress, nullptr, 0, s);
    k_macro_norm<<<1, 1024, 0, s>>>(M, rnorm);
    return cudaGetLastError();
}

// Factor, solve and apply (K and R assembled); returns the number of kernels launched.
static int macro_factor_solve_apply(const MacroDev& M, double* dFbar, int* status, cudaStream_t s) {
    int launches = 0;
    k_mstatus_clear<<<1, 1, 0, s>>>(status);
    ++launches;
    const int n = M.nfree;
    for (int j0 = 0; j0 < n; j0 += MB) {
        const int nb = std::min(MB, n - j0), j1 = j0 + nb - 1, rl = std::min(n - 1, j1 + M.kd);
        k_mchol_diag<<<1, 1024, 0, s>>>(M, j0, status);
        ++launches;
        const int m = rl - j1;
        if (m <= 0) continue;
        k_mchol_trsm<<<(m + 7) / 8, 256, 0, s>>>(M, j0);
        const int T = (m + MB - 1) / MB;
        k_mchol_update<<<T * (T + 1) / 2, 256, 0, s>>>(M, j0);
        launches += 2;
    }
    k_mchol_solve<<<1, 1024, 0, s>>>(M);
    const int g = (M.d * M.nnode + 127) / 128;
    k_macro_apply<<<g, 128, 0, s>>>(M);
    if (M.d == 3)
        k_macro_apply2<3><<<(M.ngp + 127) / 128, 128, 0, s>>>(M, dFbar);
    else
        k_macro_apply2<2><<<(M.ngp + 127) / 128, 128, 0, s>>>(M, dFbar);
    k_macro_apply3<<<g, 128, 0, s>>>(M);
    return launches + 4;
}

cudaError_t launch_macro_solve(const MacroDev& M, const double* stress, const double* Cbar, double* dFbar,
                               double* rnorm, int* status, cudaStream_t s, int* launches) {
    cudaError_t e = cudaMemsetAsync(M.K, 0, sizeof(double) * (size_t)M.nfree * (M.kd + 1), s);
    if (e != cudaSuccess) return e;
    macro_assemble(M, stress, Cbar, 1, s);
    k_macro_norm<<<1, 1024, 0, s>>>(M, rnorm);
    *launches = 2 + macro_factor_solve_apply(M, dFbar, status, s);
    return cudaGetLastError();
}

// The steps of launch_macro_solve on caller-owned K and R (the MacroDev's K and R
// pointers replaced): assemble (K only when Cbar is given) ...
cudaError_t launch_macro_assemble_only(const MacroDev& M, const double* stress, const double* Cbar, int elem,
                                       cudaStream_t s) {
    if (Cbar) {
        cudaError_t e = cudaMemsetAsync(M.K, 0, sizeof(double) * (size_t)M.nfree * (M.kd + 1), s);
        if (e != cudaSuccess) return e;
    }
    if (elem && Cbar)
        k_macro_assemble_elem<<<(2 * M.nnode + 127) / 128, 128, 0, s>>>(M, stress, Cbar);
    else
        macro_assemble(M, stress, Cbar, Cbar ? 1 : 0, s);
    return cudaGetLastError();
}

// ... the norm of R ...
cudaError_t launch_macro_norm(const MacroDev& M, double* rnorm, cudaStream_t s) {
    k_macro_norm<<<1, 1024, 0, s>>>(M, rnorm);
    return cudaGetLastError();
}

// ... and the factorisation, solve and update (K is overwritten by its factor).
cudaError_t launch_macro_factor_apply(const MacroDev& M, double* dFbar, double* rnorm, int* status, cudaStream_t s,
                                      int* launches) {
    k_macro_norm<<<1, 1024, 0, s>>>(M, rnorm);
    *launches = 1 + macro_factor_solve_apply(M, dFbar, status, s);
    return cudaGetLastError();
}

cudaError_t launch_macro_solve_elem(const MacroDev& M, const double* stress, const double* Cbar, double* dFbar,
                                    double* rnorm, int* status, cudaStream_t s, int* launches) {
    cudaError_t e = cudaMemsetAsync(M.K, 0, sizeof(double) * (size_t)M.nfree * (M.kd + 1), s);
    if (e != cudaSuccess) return e;
    k_macro_assemble_elem<<<(2 * M.nnode + 127) / 128, 128, 0, s>>>(M, stress, Cbar);
    k_macro_norm<<<1, 1024, 0, s>>>(M, rnorm);
    *launches = 2 + macro_factor_solve_apply(M, dFbar, status, s);
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
