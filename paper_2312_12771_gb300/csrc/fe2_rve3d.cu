// 3D (Hex8) RVE block and the wide-band factorisation.
//
// S1 - S3 for trilinear Hex8 elements with 2x2x2 Gauss points (Section 2.2,
// Eqs. (microdefo), (microGrad); Section 3, Eqs. (linSys3), (linSys4);
// Section 4, Eqs. (discreteSys_K/D/L)); periodic reduction with the corner
// pinned (Section 2.2, Eq. (Con)(iii); Section 5.2).  Constitutive laws in 3D:
// H = cof F (Section 2.1), P = mu F + (kappa (J-1) - mu/J) H and
// A = mu I + (mu/J^2 + kappa) H (x) H + (kappa (J-1) - mu/J) dH/dF for the
// Neo-Hooke law of Eq. (MR) with beta = 0; isotropic linear elasticity.
//
// k_band_factor_gw: the band Cholesky of S4 for bands too wide for a
// shared-memory window (3D: kd = 3 (2N^2 + 2N + 2) + 2, i.e. 440 at N = 8):
// the sliding window is L itself (columns j0 .. j0 + kd + 31 of the factor's
// output, stride kd + 1, in the launch slot's workspace, mostly in L2), so a
// finished panel needs no copy; the panel, the diagonal block and the
// right-hand-side rows (a ring of kd + 32 slots) stay in shared memory.
// Same panel algorithm as the shared-memory kernel, any dimension.  The FP32
// kernel is bounded to 128 registers so that two CTAs share an SM: the update's
// global read-modify-write latency is the limit, and a second RVE per SM hides
// part of it.
#include "fe2_internal.cuh"
#include "fe2_panel.cuh"
#include "fe2_ptx.cuh"
#include "fe2_reduce.cuh"

namespace fe2 {

namespace {

constexpr double kG = 0.57735026918962576451;  // 1/sqrt(3)
constexpr int GW_PRE = 24;  // update-block columns whose old values are staged in shared memory (FP32)

// dN_a/dX_J at Gauss point q of a cube element of side h (a, q = bx + 2 by + 4 bz)
__device__ __forceinline__ double grad3(int q, int a, int J, double h) {
    double v = 1.0 / (4.0 * h);
    for (int K = 0; K < 3; ++K) {
        const double s = ((a >> K) & 1) ? 1.0 : -1.0;
        const double xi = ((q >> K) & 1) ? kG : -kG;
        v *= (K == J) ? s : (1.0 + s * xi);
    }
    return v;
}

// The law at one Gauss point in the form A_iJkL = al d_ik d_JL + be H_iJ H_kL +
// ga H_iL H_kJ, with P.  Linear (small strain, H = I): A = lambda d_iJ d_kL +
// mu (d_ik d_JL + d_iL d_Jk).  Compressible Neo-Hooke, W = mu/2 (tr C - 3) -
// mu ln J + kappa/2 (J - 1)^2: P = mu F + s H with H = cof F = J F^-T and
// s = kappa (J - 1) - mu / J; dH_iJ/dF_kL = (H_iJ H_kL - H_iL H_kJ) / J gives
// A = mu d_ik d_JL + (c + s/J) H_iJ H_kL - (s/J) H_iL H_kJ, c = mu / J^2 + kappa.
__device__ void law3(const double* m, const double F[3][3], double& al, double& be, double& ga, double H[3][3],
                     double P[3][3]) {
    const int model = (int)m[0];
    if (model == FE2_MODEL_LINEAR) {
        const double E = m[1], nu = m[2];
        const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = E / (2.0 * (1.0 + nu));
        double eps[3][3];
        for (int i = 0; i < 3; ++i)
            for (int J = 0; J < 3; ++J) eps[i][J] = 0.5 * (F[i][J] + F[J][i]) - (i == J ? 1.0 : 0.0);
        const double tr = eps[0][0] + eps[1][1] + eps[2][2];
        for (int i = 0; i < 3; ++i)
            for (int J = 0; J < 3; ++J) {
                P[i][J] = (i == J ? lam * tr : 0.0) + 2.0 * mu * eps[i][J];
                H[i][J] = i == J ? 1.0 : 0.0;
            }
        al = mu, be = lam, ga = mu;
        return;
    }
    const double mu = m[1], kappa = m[2];
    for (int i = 0; i < 3; ++i)
        for (int J = 0; J < 3; ++J) {
            const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, J1 = (J + 1) % 3, J2 = (J + 2) % 3;
            H[i][J] = F[i1][J1] * F[i2][J2] - F[i1][J2] * F[i2][J1];
        }
    const double Jd = F[0][0] * H[0][0] + F[0][1] * H[0][1] + F[0][2] * H[0][2];
    const double s = kappa * (Jd - 1.0) - mu / Jd, c = mu / (Jd * Jd) + kappa;
    for (int i = 0; i < 3; ++i)
        for (int J = 0; J < 3; ++J) P[i][J] = mu * F[i][J] + s * H[i][J];
    al = mu, be = c + s / Jd, ga = -s / Jd;
}

// S1 + S2: the rows of every (element, local node a) written to the element
// workspace [comp][nn]: per a: kr[b][i][k] (72), f[i] (3), kM[i][kL] (27); after the
// 8 row groups: K_MM (81) and Pint (9) of the element.  A CTA holds 16 elements.
// Phase 1: the thread of each (element, Gauss point) evaluates the law once and
// caches A (81) and P (9) in shared memory.  Phase 2: one thread per (element, a,
// component i) integrates row i of node a (24 + 9 + 1 accumulators, in registers).
constexpr int E3_ELEMS = 32;  // elements per CTA of the Hex8 assembly (one per lane)
constexpr int E3_THREADS = 8 * 32;  // phase 1: warp = Gauss point; phase 2: warps share the element's blocks
constexpr int E3_C = 45;            // cached values per (Gauss point, element)

// Node pair p of the element matrix: p < 28 the pairs a < b in row order, then
// the diagonal pairs (p - 28, p - 28).
__device__ __forceinline__ void pair3(int p, int& a, int& b) {
    if (p >= 28) {
        a = b = p - 28;
        return;
    }
    a = 0;
    while (p >= 7 - a) p -= 7 - a, ++a;
    b = a + 1 + p;
}

// S1-S2 for Hex8 RVEs: a CTA takes E3_ELEMS (32) elements.
//
// Both laws give a tangent of the form A_iJkL = al d_ik d_JL + be H_iJ H_kL +
// ga H_iL H_kJ (Neo-Hooke: H = cof F, al = mu, be = c + s/J, ga = -s/J with
// P = mu F + s H; linear: H = I, al = mu, be = lambda, ga = mu).  With
// h_b = H G_b the node-pair block of the element stiffness is
//   k_e(a, b)_ik = sum_q w [al (G_a . G_b) d_ik + be h_a,i h_b,k + ga h_b,i h_a,k],
// which needs no 81-entry tangent.  The macro coupling is K_mM = k_e X (X the
// element's node coordinates relative to its first node: trilinear gradients
// reproduce linear fields, sum_b G_b (x) X_b = I at every Gauss point).
//
// Phase 1: warp q, lane = element, evaluates the law at Gauss point q and caches
// w al, w be, w ga, H, w P and h_b (element fastest).  Phase 2: the 36 node-pair
// blocks (b >= a; the gather reads k_e(b, a) as the transpose of k_e(a, b)) go to
// the warps in turn; warp w also integrates f of node w.  Gauss points are summed
// in order.  Phase 3: warp a forms the K_mM rows of node a from the finished
// blocks.  Phase 4: K_MM and Pint from those rows and f (the same identity).
__global__ void __launch_bounds__(E3_THREADS, 2) k_assemble_elems3(const RveDev* __restrict__ tab,
                                                                   const int* __restrict__ ids,
                                                                   const double* __restrict__ Fbar) {
    extern __shared__ __align__(16) double cache3[];  // [8 GP][E3_C][E3_ELEMS]
    __shared__ double Gt[8][8][3];                     // [GP][node][J]
    __shared__ double Dg[8][8][8];                     // [GP][a][b]: G_a . G_b
    const RveDev r = tab[ids[blockIdx.y]];
    const int N = r.N, nn = r.nn;
    const double h = 1.0 / N, wq = 0.125 * h * h * h;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int k = tid; k < 8 * 8 * 3; k += blockDim.x) {
        const int q = k / 24, b = (k / 3) % 8, J = k % 3;
        Gt[q][b][J] = grad3(q, b, J, h);
    }
    for (int k = tid; k < 8 * 8 * 8; k += blockDim.x) {
        const int q = k / 64, a = (k / 8) % 8, b = k % 8;
        double d = 0.0;
        for (int J = 0; J < 3; ++J) d += grad3(q, a, J, h) * grad3(q, b, J, h);
        Dg[q][a][b] = d;
    }
    double Fb[9];
    for (int k = 0; k < 9; ++k) Fb[k] = Fbar[9 * blockIdx.y + k];
    __syncthreads();
    const int el = lane, e = blockIdx.x * E3_ELEMS + el;
    // phase 1: the law of element el at Gauss point q = warp
    if (e < nn) {
        const int q = warp;
        const int ex = e % N, ey = (e / N) % N, ez = e / (N * N);
        double F[3][3];
        for (int i = 0; i < 3; ++i)
            for (int J = 0; J < 3; ++J) F[i][J] = Fb[3 * i + J];
        for (int b = 0; b < 8; ++b) {
            const int i = (ex + (b & 1)) % N, j = (ey + ((b >> 1) & 1)) % N, k = (ez + (b >> 2)) % N;
            const int qn = fold_pos(i, N) + N * fold_pos(j, N) + N * N * fold_pos(k, N);
            for (int c = 0; c < 3; ++c) {
                const double w = (qn == 0 || r.zero_w) ? 0.0 : r.w[3 * (qn - 1) + c];
                for (int J = 0; J < 3; ++J) F[c][J] += w * Gt[q][b][J];
            }
        }
        double al, be, ga, H[3][3], P[3][3];
        law3(r.mat + 4 * r.phase[e], F, al, be, ga, H, P);
        double* c = cache3 + (size_t)q * E3_C * E3_ELEMS + el;
        c[0] = wq * al;
        c[E3_ELEMS] = wq * be;
        c[2 * E3_ELEMS] = wq * ga;
        for (int k = 0; k < 9; ++k) c[(3 + k) * E3_ELEMS] = H[k / 3][k % 3];
        for (int k = 0; k < 9; ++k) c[(12 + k) * E3_ELEMS] = wq * P[k / 3][k % 3];
        for (int b = 0; b < 8; ++b)
            for (int i = 0; i < 3; ++i)
                c[(21 + 3 * b + i) * E3_ELEMS] = H[i][0] * Gt[q][b][0] + H[i][1] * Gt[q][b][1] + H[i][2] * Gt[q][b][2];
    }
    __syncthreads();
    // lanes past the last element take no part below but reach every barrier
    const bool live = e < nn;
    constexpr int RC = elem_row_comps(3);
    double* E = r.elem;
    const double* ce = cache3 + el;
    // node-pair blocks k_e(a, b), b >= a
    for (int p = warp; live && p < 36; p += 8) {
        int a, b;
        pair3(p, a, b);
        double acc[9], dacc = 0.0;
#pragma unroll
        for (int t = 0; t < 9; ++t) acc[t] = 0.0;
#pragma unroll 1
        for (int q = 0; q < 8; ++q) {
            const double* c = ce + (size_t)q * E3_C * E3_ELEMS;
            const double al = c[0], be = c[E3_ELEMS], ga = c[2 * E3_ELEMS];
            double ha[3], hb[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                ha[i] = c[(21 + 3 * a + i) * E3_ELEMS];
                hb[i] = c[(21 + 3 * b + i) * E3_ELEMS];
            }
            dacc += al * Dg[q][a][b];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const double bha = be * ha[i], ghb = ga * hb[i];
#pragma unroll
                for (int k = 0; k < 3; ++k) acc[3 * i + k] = __fma_rn(ghb, ha[k], __fma_rn(bha, hb[k], acc[3 * i + k]));
            }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                E[(size_t)(a * RC + 9 * b + 3 * i + k) * nn + e] = i == k ? acc[3 * i + k] + dacc : acc[3 * i + k];
    }
    // f of node a = warp: sum_q w P G_a
    if (live) {
        const int a = warp;
        double f[3] = {0.0, 0.0, 0.0};
#pragma unroll 1
        for (int q = 0; q < 8; ++q) {
            const double* c = ce + (size_t)q * E3_C * E3_ELEMS;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int J = 0; J < 3; ++J) f[i] += c[(12 + 3 * i + J) * E3_ELEMS] * Gt[q][a][J];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) E[(size_t)(a * RC + 72 + i) * nn + e] = f[i];
    }
    // phase 3: K_mM rows of node a = warp, k_e(a, .) X = h sum_{b: bit L of b} k_e(a, b), from the
    // blocks written above (this CTA's global writes are visible after the barrier)
    __syncthreads();
    if (live) {
        const int a = warp;
#pragma unroll 1
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                double v[8];
#pragma unroll
                for (int b = 0; b < 8; ++b)
                    v[b] = b >= a ? E[(size_t)(a * RC + 9 * b + 3 * i + k) * nn + e]
                                  : E[(size_t)(b * RC + 9 * a + 3 * k + i) * nn + e];
                const double sx = (v[1] + v[3]) + (v[5] + v[7]), sy = (v[2] + v[3]) + (v[6] + v[7]),
                             sz = (v[4] + v[5]) + (v[6] + v[7]);
                const size_t o = (size_t)(a * RC + 75 + 9 * i + 3 * k) * nn + e;
                E[o] = h * sx;
                E[o + nn] = h * sy;
                E[o + 2 * (size_t)nn] = h * sz;
            }
    }
    // phase 4: K_MM = X^T k_e X and Pint = sum_a f_a (x) X_a, from the finished rows:
    // K_MM[(i, J)][(k, L)] = h sum_{a: bit J of a} K_mM[a][i][(k, L)], Pint[(i, J)] likewise
    // from f_a; entry t = 9 m + n (t < 81) or Pint m = t - 81 on warp t % 8
    __syncthreads();
    if (live) {
        for (int t = warp; t < 90; t += 8) {
            const int m = t < 81 ? t / 9 : t - 81, i = m / 3, J = m % 3;
            const int col = t < 81 ? 75 + 9 * i + t % 9 : 72 + i;
            double sum = 0.0;
#pragma unroll
            for (int a = 0; a < 8; ++a)
                if ((a >> J) & 1) sum += E[(size_t)(a * RC + col) * nn + e];
            E[(size_t)(8 * RC + t) * nn + e] = h * sum;
        }
    }
}

// S3: node-row gather through the periodic map (one CTA per RVE).  Each node row
// is owned by one thread (deterministic order): per neighbour block off, the 9
// entries are summed over the elements around the node in the order of their
// local node a (k_e(a, b) with b < a read as the transpose of k_e(b, a)) and
// stored once.  K_MM and Pint are summed over elements by one thread per component.
__global__ void __launch_bounds__(256) k_reduce3(const RveDev* __restrict__ tab, const int* __restrict__ ids) {
    const RveDev r = tab[ids[blockIdx.x]];
    const int N = r.N, nn = r.nn, RC = elem_row_comps(3);
    const double* __restrict__ E = r.elem;
    double* __restrict__ st = r.stencil;
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
        const int i = unfold_pos(q % N, N), j = unfold_pos((q / N) % N, N), k = unfold_pos(q / (N * N), N);
        int ea[8];  // the element whose local node a is node q
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
            ea[a] = (i - ax + N) % N + N * ((j - ay + N) % N) + N * N * ((k - az + N) % N);
        }
        for (int off = 0; off < 27; ++off) {
            const int ox = off % 3 - 1, oy = (off / 3) % 3 - 1, oz = off / 9 - 1;  // b - a per direction
            double acc[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) acc[t] = 0.0;
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const int bx = (a & 1) + ox, by = ((a >> 1) & 1) + oy, bz = (a >> 2) + oz;
                if (bx < 0 || bx > 1 || by < 0 || by > 1 || bz < 0 || bz > 1) continue;
                const int b = bx + 2 * by + 4 * bz, e = ea[a];
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int c2 = 0; c2 < 3; ++c2) {
                        const int comp = b >= a ? a * RC + 9 * b + 3 * c + c2 : b * RC + 9 * a + 3 * c2 + c;
                        acc[3 * c + c2] += E[(size_t)comp * nn + e];
                    }
            }
#pragma unroll
            for (int t = 0; t < 9; ++t) st[(size_t)(off * 9 + t) * nn + q] = acc[t];
        }
        if (q != 0) {
            double f[3] = {0.0, 0.0, 0.0}, kM[3][9];
            for (int c = 0; c < 3; ++c)
                for (int kL = 0; kL < 9; ++kL) kM[c][kL] = 0.0;
            for (int a = 0; a < 8; ++a) {
                const int e = ea[a];
                int c0 = a * RC + 72;
                for (int c = 0; c < 3; ++c) f[c] += E[(size_t)(c0++) * nn + e];
                for (int c = 0; c < 3; ++c)
                    for (int kL = 0; kL < 9; ++kL) kM[c][kL] += E[(size_t)(c0++) * nn + e];
            }
            for (int c = 0; c < 3; ++c) {
                const int dof = 3 * (q - 1) + c;
                for (int kL = 0; kL < 9; ++kL) r.rhs[(size_t)kL * r.nm + dof] = kM[c][kL];
                r.rhs[(size_t)9 * r.nm + dof] = f[c];
            }
        }
    }
    if (threadIdx.x < 90) {
        double s = 0.0;
        for (int e = 0; e < nn; ++e) s += E[(size_t)(8 * RC + threadIdx.x) * nn + e];
        if (threadIdx.x < 81)
            r.KMM[threadIdx.x] = s;
        else
            r.Pint[threadIdx.x - 81] = s;
    }
}

// FP64 residual R = [K_mM | r_m] - K_mm X (3D stencil, 27 neighbour blocks)
__global__ void __launch_bounds__(128) k_residual3(const RveDev* __restrict__ tab, const int* __restrict__ ids,
                                                   Workspace ws, const int* __restrict__ active) {
    if (active && !active[blockIdx.y]) return;
    const RveDev r = tab[ids[blockIdx.y]];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= r.nn || q == 0) return;
    const int nn = r.nn, nm = r.nm;
    double* R = (double*)(ws.base + blockIdx.y * ws.stride + ws.offR);
    double acc[3][10];
    for (int c = 0; c < 3; ++c)
        for (int rr = 0; rr < 10; ++rr) acc[c][rr] = 0.0;
    for (int off = 0; off < 27; ++off) {
        const int qn = r.nbr[q * 27 + off];
        if (qn == 0) continue;
        for (int c = 0; c < 3; ++c)
            for (int c2 = 0; c2 < 3; ++c2) {
                const double kv = r.stencil[(size_t)((off * 3 + c) * 3 + c2) * nn + q];
                for (int rr = 0; rr < 10; ++rr) acc[c][rr] += kv * r.X[(size_t)rr * nm + 3 * (qn - 1) + c2];
            }
    }
    for (int c = 0; c < 3; ++c) {
        const int dof = 3 * (q - 1) + c;
        for (int rr = 0; rr < 10; ++rr) R[(size_t)rr * nm + dof] = r.rhs[(size_t)rr * nm + dof] - acc[c][rr];
    }
}

// One CTA per RVE (3D: d^2 = 9, nr = 10): G1 = rhs_M^T X (9 x 10) and G2 = X'_M^T R
// (9 x 10, X' = X + dx on the second-order pass, corrected = 2), in three passes over
// the macro components, three at a time: every thread keeps 60 partial sums over its
// DOFs in registers and the CTA adds them (cta_sum).  The epilogue runs on 90 threads,
// the norms of the error estimate meet in one more CTA sum.
__global__ void __launch_bounds__(256) k_schur3(const RveDev* __restrict__ tab, const int* __restrict__ ids,
                                                Workspace ws, int corrected, double* __restrict__ sigma,
                                                double* __restrict__ Cbar, int* __restrict__ status,
                                                double* __restrict__ err, const double* __restrict__ tol,
                                                int* __restrict__ redo, int only_flagged, int final_sweep) {
    constexpr int AC = 3, NV = 2 * AC * 10;
    __shared__ double red[NV * 33];
    __shared__ double tp[NV];
    __shared__ double tot[183];
    if (only_flagged && !redo[blockIdx.x]) return;
    const RveDev r = tab[ids[blockIdx.x]];
    const int nm = r.nm, nmp = r.nm_pad;
    const double* R = (const double*)(ws.base + blockIdx.x * ws.stride + ws.offR);
    // corrected = 2: the FP32 correction dx of every column in the slot's y region;
    // the correction term uses X' = X + dx (as in the 2D kernel), X' is stored
    const float* dX = (const float*)(ws.base + blockIdx.x * ws.stride + ws.offY);
    const int tid = threadIdx.x;
    for (int a0 = 0; a0 < 9; a0 += AC) {
        double acc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = 0.0;
        for (int m = tid; m < nm; m += blockDim.x) {
            double ra[AC], xa[AC];
#pragma unroll
            for (int q = 0; q < AC; ++q) {
                ra[q] = r.rhs[(size_t)(a0 + q) * nm + m];
                double x = r.X[(size_t)(a0 + q) * nm + m];
                if (corrected == 2) x += (double)dX[(size_t)(a0 + q) * nmp + m];
                xa[q] = x;
            }
#pragma unroll
            for (int b = 0; b < 10; ++b) {
                const double xb = r.X[(size_t)b * nm + m];
#pragma unroll
                for (int q = 0; q < AC; ++q) acc[q * 10 + b] += ra[q] * xb;
                if (corrected) {
                    const double rb = R[(size_t)b * nm + m];
#pragma unroll
                    for (int q = 0; q < AC; ++q) acc[AC * 10 + q * 10 + b] += xa[q] * rb;
                }
            }
        }
        cta_sum<NV>(acc, red, tp);
        if (tid < NV) {
            const int w = tid / (AC * 10), q = (tid / 10) % AC, b = tid % 10;
            tot[w * 90 + (a0 + q) * 10 + b] = tp[tid];
        }
    }
    if (corrected == 2) {
        double ex[3] = {0.0, 0.0, 0.0};
        for (int m = tid; m < nm; m += blockDim.x)
            for (int c = 0; c < 9; ++c) {
                const double dx = (double)dX[(size_t)c * nmp + m];
                const double x = r.X[(size_t)c * nm + m];
                ex[0] += dx * R[(size_t)c * nm + m];
                ex[1] += dx * dx;
                ex[2] += x * x;
            }
        cta_sum<3>(ex, red, tot + 180);
        for (int k = tid; k < 10 * nm; k += blockDim.x) {
            const int c = k / nm, m = k - c * nm;
            r.X[k] += (double)dX[(size_t)c * nmp + m];
        }
    }
    __syncthreads();
    // thread t < 81: Cbar entry (a, b) = (t / 9, t % 9); 81 <= t < 90: sigma_eff component
    double nv[2] = {0.0, 0.0};
    int bad = 0;
    if (tid < 81) {
        const int a = tid / 9, b = tid % 9;
        double v = r.KMM[tid] - tot[a * 10 + b];
        if (corrected) {
            const double g = tot[90 + a * 10 + b];
            v -= g;
            nv[1] = g * g;
        }
        nv[0] = v * v;
        bad = !isfinite(v);
        Cbar[(size_t)blockIdx.x * 81 + tid] = v;
    } else if (tid < 90) {
        const int a = tid - 81;
        double sg = r.Pint[a] - tot[a * 10 + 9];
        if (corrected) sg -= tot[90 + a * 10 + 9];
        bad = !isfinite(sg);
        sigma[(size_t)blockIdx.x * 9 + a] = sg;
    }
    bad = __syncthreads_or(bad);
    cta_sum<2>(nv, red, tp);
    if (tid == 0) {
        const double cn = tp[0], corr = tp[1];
        double e = 0.0;
        if (corrected == 1) e = corr / fmax(cn, 1e-300);
        if (corrected == 2) e = fabs(tot[180]) / sqrt(fmax(cn, 1e-300)) * sqrt(tot[181] / fmax(tot[182], 1e-300));
        if (err) err[blockIdx.x] = e;
        if (bad && status[blockIdx.x] == FE2_OK) status[blockIdx.x] = FE2_ERR_NAN;
        const bool over = corrected && !(e <= *tol);
        if (redo) redo[blockIdx.x] = (over && status[blockIdx.x] == FE2_OK) ? 1 : 0;
        if (final_sweep && over && status[blockIdx.x] == FE2_OK) status[blockIdx.x] = FE2_ERR_NO_CONV;
    }
}

__device__ __forceinline__ int wrapS3(int x, int S) { return x >= S ? x - S : x; }

// four consecutive shared-memory values (16-byte aligned) in one or two vector loads
template <typename T>
struct Ld4;
template <>
struct Ld4<double> {
    __device__ __forceinline__ static void load(const double* p, double* o) {
        const double2 v0 = *reinterpret_cast<const double2*>(p), v1 = *reinterpret_cast<const double2*>(p + 2);
        o[0] = v0.x, o[1] = v0.y, o[2] = v1.x, o[3] = v1.y;
    }
};

template <typename T>
struct GwLayout {
    int kd, S, LDW, KR, KP, nr, nblk;
    size_t offBw, offDinv, offBlk, offL11, offOld, total;
    __host__ __device__ void init(int kd_, int nr_) {
        kd = kd_;
        nr = nr_;
        S = kd + NB;
        LDW = kd + 1;
        KR = kd + nr;
        KP = (KR + 31) & ~31;
        const int RB = KP / 32, CB = (kd + 31) / 32;
        nblk = 0;
        for (int K = 0; K < CB; ++K) nblk += RB - K;
        size_t o = (size_t)NB * KP * sizeof(T);  // Pn
        offBw = o;
        o += (size_t)nr * S * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offDinv = o;
        o += 2 * NB * sizeof(T);  // dinv, then one column of the diagonal block
        o = (o + 15) & ~(size_t)15;
        offBlk = o;
        o += (size_t)nblk * 4;
        o = (o + 15) & ~(size_t)15;
        offL11 = o;  // packed L11 (fe2_panel.cuh)
        o += (size_t)L11P_LEN * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offOld = o;  // FP32: per warp, old window values of GW_PRE columns of its update block
        if (sizeof(T) == 4) o += (size_t)(FACT_THREADS / 32) * GW_PRE * NB * sizeof(T);
        total = (o + 15) & ~(size_t)15;
    }
};

// Columns [c0, c0 + ncol) of K_mm into their columns of L (stride LDW), one
// (column, neighbour) pair per item, items t0, t0 + nt, ...; the columns must be
// zero.  The neighbours of a node are distinct for N >= 3, so no two items write
// the same entry.  Columns in [nm, nmp) get a unit diagonal; none exist beyond.
template <typename T>
__device__ __forceinline__ void gw_load_columns(T* __restrict__ Lw, int LDW, int c0, int ncol, int nmp,
                                                const RveDev& r, int t0, int nt) {
    const int d = r.d, ns = d == 2 ? 9 : 27, nn = r.nn, nm = r.nm;
    for (int p = t0; p < ncol * ns; p += nt) {
        const int x = p / ns, off = p - x * ns, c = c0 + x;
        if (c >= nmp) continue;
        T* Wc = Lw + (size_t)c * LDW;
        if (c >= nm) {
            if (off == 0) Wc[0] = T(1);
            continue;
        }
        const int q = c / d + 1, cc = c - d * (q - 1);
        const int qn = r.nbr[q * ns + off];
        if (qn == 0) continue;
        for (int c2 = 0; c2 < d; ++c2) {
            const int row = d * (qn - 1) + c2;
            if (row >= c) Wc[row - c] += (T)r.stencil[(size_t)((off * d + cc) * d + c2) * nn + q];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(FACT_THREADS, sizeof(T) == 4 ? 2 : 1) k_band_factor_gw(const RveDev* __restrict__ tab,
                                                                 const int* __restrict__ ids, Workspace ws,
                                                                 int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const RveDev r = tab[ids[blockIdx.x]];
    GwLayout<T> lay;
    lay.init(r.kd, r.nr);
    const int kd = lay.kd, S = lay.S, LDW = lay.LDW, KR = lay.KR, KP = lay.KP, nr = lay.nr;
    const int nmp = r.nm_pad, nm = r.nm;
    T* Pn = (T*)smem;
    T* Bw = (T*)(smem + lay.offBw);
    T* dinv = (T*)(smem + lay.offDinv);
    unsigned* blk = (unsigned*)(smem + lay.offBlk);
    T* L11p = (T*)(smem + lay.offL11);
    __shared__ int s_bad;
    char* slot = ws.base + blockIdx.x * ws.stride;
    T* Lg = (T*)slot;
    T* Yg = (T*)(slot + ws.offY);
    T* Dg = (T*)(slot + ws.offD);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    T* Old = (T*)(smem + lay.offOld) + (size_t)warp * GW_PRE * NB;  // FP32 only: [column w][lane]
    if (tid == 0) {
        s_bad = 0;
        const int RB = KP / 32, CB = (kd + 31) / 32;
        int x = 0;
        for (int K = 0; K < CB; ++K)
            for (int I = K; I < RB; ++I) blk[x++] = (unsigned)I | ((unsigned)K << 16);
    }
    for (int k = tid; k < NB * KP; k += blockDim.x) Pn[k] = T(0);
    for (size_t k = tid; k < (size_t)min(S, nmp) * LDW; k += blockDim.x) Lg[k] = T(0);
    for (int k = tid; k < nr * S; k += blockDim.x) {
        const int rr = k / S, c = k - rr * S;
        Bw[k] = (c < nm && c < kd) ? (T)r.rhs[(size_t)rr * nm + c] : T(0);
    }
    __syncthreads();
    gw_load_columns<T>(Lg, LDW, 0, min(kd, nmp), nmp, r, tid, blockDim.x);
    __syncthreads();
    int base = 0;
    for (int j0 = 0; j0 < nmp; j0 += NB) {
        // 1: diagonal block (warp 0) / entering columns [j0+kd, j0+kd+NB) (other warps)
        if (warp == 0) {
            T a[NB];
#pragma unroll
            for (int c = 0; c < NB; ++c)
                a[c] = (c <= lane && lane - c <= kd) ? Lg[(size_t)(j0 + c) * LDW + (lane - c)] : T(0);
            int badb = 0;
            chol_block_steps<T, 0>(a, lane, dinv, badb);
            if (lane == 0 && badb) s_bad = 1;
            __syncwarp();
#pragma unroll
            for (int c = 0; c < NB; ++c)
                if (c <= lane && lane - c <= kd) Lg[(size_t)(j0 + c) * LDW + (lane - c)] = a[c];
            const T dl = dinv[lane];
            Dg[j0 + lane] = dl;
            diag_pack<T>(a, dl, L11p, lane);
        } else {
            const int nt = blockDim.x - 32, t0 = tid - 32;
            for (int x = warp - 1; x < NB; x += nwarps - 1) {
                if (j0 + kd + x >= nmp) break;
                T* Wc = Lg + (size_t)(j0 + kd + x) * LDW;
                for (int off = lane; off < LDW; off += 32) Wc[off] = T(0);
            }
            asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
            gw_load_columns<T>(Lg, LDW, j0 + kd, NB, nmp, r, t0, nt);
            for (int p = t0; p < nr * NB; p += nt) {
                const int rr = p / NB, x = p - rr * NB, cn = j0 + kd + x;
                Bw[rr * S + wrapS3(base + kd + x, S)] = (cn < nm) ? (T)r.rhs[(size_t)rr * nm + cn] : T(0);
            }
        }
        __syncthreads();
        // 2: panel rows (L21, y)
        for (int t = tid; t < KR; t += blockDim.x) {
            T v[NB];
            if (t < kd) {
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    const int off = NB + t - c;
                    v[c] = (off <= kd) ? Lg[(size_t)(j0 + c) * LDW + off] : T(0);
                }
            } else {
#pragma unroll
                for (int c = 0; c < NB; ++c) v[c] = Bw[(t - kd) * S + wrapS3(base + c, S)];
            }
            panel_row_steps<T, 0>(v, L11p);
#pragma unroll
            for (int c = 0; c < NB; ++c) Pn[c * KP + t] = v[c];
            if (t < kd) {
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    const int off = NB + t - c;
                    if (off <= kd) Lg[(size_t)(j0 + c) * LDW + off] = v[c];
                }
            } else {
#pragma unroll
                for (int c = 0; c < NB; ++c) Bw[(t - kd) * S + wrapS3(base + c, S)] = v[c];
            }
        }
        __syncthreads();
        // 3: rank-NB update (32x32 warp blocks) and stream out the finished panel
        {
            // lane = row t1 = 32I + lane of the block, 32 columns t2 = 32K + w per lane:
            // every write-back step is one coalesced 128-byte row segment of a window
            // column in global memory; a warp loads all old values before storing any
            for (int b = warp; b < lay.nblk; b += nwarps) {
                const unsigned bv = blk[b];
                const int I = bv & 0xffff, K = bv >> 16;
                const int t1 = 32 * I + lane, q0 = 32 * K;
                const bool fast = I > K && 32 * I + 32 <= kd && q0 + 32 <= kd && j0 + NB + q0 + 32 <= nmp;
                T* Lq = Lg + (size_t)(j0 + NB + q0) * LDW;  // column t2 = q0 + w at Lq + w LDW
                T oldr[NB - GW_PRE];
                if constexpr (sizeof(T) == 4) {
                    // the old window values of this lane's entries (row t1 < kd, column
                    // t2 <= t1, t2 < kd) travel while the products accumulate: GW_PRE
                    // columns to shared memory, the rest to registers
#pragma unroll 8
                    for (int w = 0; w < GW_PRE; ++w) {
                        const int t2 = q0 + w;
                        if (t2 < kd && t1 >= t2 && t1 < kd && j0 + NB + t2 < nmp)
                            cp_async4(Old + w * NB + lane, Lq + (size_t)w * LDW + (t1 - t2));
                    }
                    cp_async_commit();
#pragma unroll
                    for (int w = GW_PRE; w < NB; ++w) {
                        const int t2 = q0 + w;
                        oldr[w - GW_PRE] = (t2 < kd && t1 >= t2 && t1 < kd && j0 + NB + t2 < nmp)
                                               ? Lq[(size_t)w * LDW + (t1 - t2)] : T(0);
                    }
                }
                T acc[32];
                if constexpr (sizeof(T) == 4) {
                    // column pairs through the paired FP32 FMA: the same roundings as
                    // two scalar FMAs in half the instructions
                    float2 acc2[16];
#pragma unroll
                    for (int w = 0; w < 16; ++w) acc2[w] = make_float2(0.f, 0.f);
#pragma unroll 2
                    for (int c = 0; c < NB; ++c) {
                        const float* pc = Pn + c * KP;
                        const float av = pc[t1];
                        const float2 a2 = make_float2(av, av);
#pragma unroll
                        for (int w4 = 0; w4 < 8; ++w4) {
                            const float4 b4 = *reinterpret_cast<const float4*>(pc + q0 + 4 * w4);
                            acc2[2 * w4] = __ffma2_rn(a2, make_float2(b4.x, b4.y), acc2[2 * w4]);
                            acc2[2 * w4 + 1] = __ffma2_rn(a2, make_float2(b4.z, b4.w), acc2[2 * w4 + 1]);
                        }
                    }
#pragma unroll
                    for (int w = 0; w < 16; ++w) acc[2 * w] = acc2[w].x, acc[2 * w + 1] = acc2[w].y;
                } else {
#pragma unroll
                    for (int w = 0; w < 32; ++w) acc[w] = T(0);
#pragma unroll 2
                    for (int c = 0; c < NB; ++c) {
                        const T* pc = Pn + c * KP;
                        const T av = pc[t1];
#pragma unroll
                        for (int w4 = 0; w4 < 8; ++w4) {
                            T bb[4];
                            Ld4<T>::load(pc + q0 + 4 * w4, bb);
#pragma unroll
                            for (int x = 0; x < 4; ++x) acc[4 * w4 + x] += av * bb[x];
                        }
                    }
                }
                if constexpr (sizeof(T) == 4) {
                    cp_async_wait_all();  // this lane's own copies: no exchange between lanes
#pragma unroll
                    for (int w = 0; w < NB; ++w) {
                        const int t2 = q0 + w;
                        if (t2 >= kd || t1 < t2 || t1 >= KR) continue;
                        if (t1 < kd) {
                            if (j0 + NB + t2 < nmp)
                                Lq[(size_t)w * LDW + (t1 - t2)] = (w < GW_PRE ? Old[w * NB + lane] : oldr[w - GW_PRE]) - acc[w];
                        } else {
                            Bw[(t1 - kd) * S + wrapS3(base + NB + t2, S)] -= acc[w];
                        }
                    }
                } else if (fast) {
                    T old[32];
#pragma unroll
                    for (int w = 0; w < 32; ++w) old[w] = Lq[(size_t)w * LDW + (t1 - (q0 + w))];
#pragma unroll
                    for (int w = 0; w < 32; ++w) Lq[(size_t)w * LDW + (t1 - (q0 + w))] = old[w] - acc[w];
                } else {
#pragma unroll
                    for (int w = 0; w < 32; ++w) {
                        const int t2 = q0 + w;
                        if (t2 >= kd || t1 < t2 || t1 >= KR) continue;
                        if (t1 < kd) {
                            if (j0 + NB + t2 < nmp) Lq[(size_t)w * LDW + (t1 - t2)] -= acc[w];
                        } else {
                            Bw[(t1 - kd) * S + wrapS3(base + NB + t2, S)] -= acc[w];
                        }
                    }
                }
            }
            for (int k = tid; k < nr * NB; k += blockDim.x) {
                const int rr = k / NB, c = k - rr * NB;
                Yg[(size_t)rr * nmp + j0 + c] = Bw[rr * S + wrapS3(base + c, S)];
            }
        }
        __syncthreads();
        base = wrapS3(base + NB, S);
    }
    if (tid == 0 && s_bad && status[blockIdx.x] == FE2_OK) status[blockIdx.x] = FE2_ERR_NOT_PD;
}

}  // namespace

cudaError_t launch_assemble_elems3(const RveDev* tab, const int* ids, int n, const double* Fbar, int maxN,
                                   cudaStream_t s) {
    const size_t smem = (size_t)E3_ELEMS * 8 * E3_C * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_assemble_elems3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((maxN * maxN * maxN + E3_ELEMS - 1) / E3_ELEMS, n);
    k_assemble_elems3<<<grid, E3_THREADS, smem, s>>>(tab, ids, Fbar);
    return cudaGetLastError();
}

cudaError_t launch_reduce3(const RveDev* tab, const int* ids, int n, cudaStream_t s) {
    k_reduce3<<<n, 256, 0, s>>>(tab, ids);
    return cudaGetLastError();
}

cudaError_t launch_residual3(const RveDev* tab, const int* ids, int n, Workspace ws, int maxnn, const int* active,
                             cudaStream_t s) {
    dim3 grid((maxnn + 127) / 128, n);
    k_residual3<<<grid, 128, 0, s>>>(tab, ids, ws, active);
    return cudaGetLastError();
}

cudaError_t launch_schur3(const RveDev* tab, const int* ids, int n, Workspace ws, int corrected, double* sigma,
                          double* Cbar, int* status, double* err, const double* tol, int* redo, cudaStream_t s,
                          int refine_sweep) {
    k_schur3<<<n, 256, 0, s>>>(tab, ids, ws, corrected, sigma, Cbar, status, err, tol, redo,
                               refine_sweep == 1 || refine_sweep == 2, refine_sweep >= 2);
    return cudaGetLastError();
}

size_t factor_gw_smem_bytes(int kd, int nr, bool fp64) {
    if (fp64) {
        GwLayout<double> l;
        l.init(kd, nr);
        return l.total;
    }
    GwLayout<float> l;
    l.init(kd, nr);
    return l.total;
}

template <typename T>
cudaError_t launch_factor_gw(const RveDev* tab, const int* ids, int n, Workspace ws, int* status, int maxkd,
                             int maxnr, cudaStream_t s) {
    GwLayout<T> lay;
    lay.init(maxkd, maxnr);
    cudaError_t e = cudaFuncSetAttribute(k_band_factor_gw<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
    if (e != cudaSuccess) return e;
    k_band_factor_gw<T><<<n, FACT_THREADS, lay.total, s>>>(tab, ids, ws, status);
    return cudaGetLastError();
}

template cudaError_t launch_factor_gw<float>(const RveDev*, const int*, int, Workspace, int*, int, int, cudaStream_t);
template cudaError_t launch_factor_gw<double>(const RveDev*, const int*, int, Workspace, int*, int, int, cudaStream_t);

}  // namespace fe2
