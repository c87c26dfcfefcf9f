// W-kernel table generation on the device, in FP64.
//
// W-projection (Section 1.7.1, from Eq. (v00) of Section 1.3) merges the
// convolution with Gbar_w = F[exp(+j 2 pi w (n - 1))] into the gridding
// convolution function; the anti-aliasing taper is the prolate spheroidal
// function (Section 2.3.4) and the function is stored beta-oversampled for
// nearest-neighbour lookup (Section 2.3.6).  For plane p:
//
//   K_p(du, dv) = int int_{[-1,1]^2} T(a) T(b) exp(+j 2 pi w_p (n - 1))
//                  exp(-j pi (du a + dv b)) da db,
//   n = sqrt(1 - (L/2)^2 (a^2 + b^2)),  T = psi_0(c, .),  c = pi S_min / 2,
//
// with a, b the field coordinates scaled to [-1, 1].  The integrand is even
// in a and in b, so with Gauss-Legendre nodes (symmetric) the transform is a
// cosine transform over the non-negative half of the nodes:
//   K_p(du, dv) = sum_{j, i >= 0} m_j m_i Tw_j Tw_i screen_ji cos(pi du a_i) cos(pi dv a_j)
// (m = 2 for a node > 0, 1 for the centre node), computed as two dense FP64
// products.  Entries are sampled at du = t_u - o_u / beta, dv = t_v - o_v / beta,
// scaled once so that the w = 0, o = 0 slice sums to 1, and stored as float2
// (and, for 16-bit storage, rounded once from FP64 to bfloat16 or float16).
//
// psi_0 comes from its Legendre expansion: the smallest eigenpair of the
// symmetric tridiagonal matrix of the prolate operator in the normalised
// even Legendre basis, found by Sturm-sequence bisection and inverse
// iteration on the (positive definite) shifted matrix.
#include "gw_internal.cuh"

#include <cmath>
#include <vector>

namespace gw {

int quad_nodes(double field, double w, int support, int smin) {
    const double half = 0.5 * field;
    const double n_min = std::sqrt(1.0 - 2.0 * half * half);
    const int h = (support - 1) / 2;
    const double c = M_PI * (double)smin / 2.0;
    const double kappa = 2.0 * M_PI * std::fabs(w) * half * half / n_min + M_PI * (h + 0.5) + c;
    return (int)std::ceil(0.75 * kappa) + 40;
}

namespace {

constexpr int kMaxTerms = 512;

__device__ double leg_a(double n) { return n / sqrt(4.0 * n * n - 1.0); }

// Smallest eigenpair of the prolate matrix; writes plain-Legendre
// coefficients coef[k] of P_{2k} (psi_0 = sum coef[k] P_{2k}), unit L2 norm,
// psi_0(0) > 0.  Single thread.
__global__ void k_pswf(double c, int K, double* __restrict__ coef, double* __restrict__ chi_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a[kMaxTerms], b[kMaxTerms], x[kMaxTerms], dd[kMaxTerms], ll[kMaxTerms];
    const double c2 = c * c;
    for (int k = 0; k < K; ++k) {
        const double n = 2.0 * k;
        const double an = (k > 0) ? leg_a(n) : 0.0;
        const double an1 = leg_a(n + 1.0);
        a[k] = n * (n + 1.0) + c2 * (an1 * an1 + an * an);
        b[k] = (k + 1 < K) ? c2 * an1 * leg_a(n + 2.0) : 0.0;
    }
    // Gershgorin interval
    double lo = a[0] - fabs(b[0]), hi = a[0] + fabs(b[0]);
    for (int k = 1; k < K; ++k) {
        const double r = fabs(b[k - 1]) + fabs(b[k]);
        lo = fmin(lo, a[k] - r);
        hi = fmax(hi, a[k] + r);
    }
    // bisection on the number of eigenvalues below x (Sturm count)
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        int cnt = 0;
        double q = a[0] - mid;
        if (q == 0.0) q = -1e-300;
        cnt += q < 0.0;
        for (int k = 1; k < K; ++k) {
            q = (a[k] - mid) - b[k - 1] * b[k - 1] / q;
            if (q == 0.0) q = -1e-300;
            cnt += q < 0.0;
        }
        if (cnt >= 1) hi = mid; else lo = mid;
    }
    *chi_out = 0.5 * (lo + hi);
    // inverse iteration with shift lo (below chi_0: the shifted matrix is
    // positive definite, so the LDL^T solve needs no pivoting)
    const double sigma = lo - 1e-12 * fmax(1.0, fabs(lo));
    dd[0] = a[0] - sigma;
    for (int k = 1; k < K; ++k) {
        ll[k] = b[k - 1] / dd[k - 1];
        dd[k] = (a[k] - sigma) - ll[k] * b[k - 1];
    }
    for (int k = 0; k < K; ++k) x[k] = 1.0;
    for (int it = 0; it < 6; ++it) {
        for (int k = 1; k < K; ++k) x[k] -= ll[k] * x[k - 1];          // L y = x
        for (int k = 0; k < K; ++k) x[k] /= dd[k];                      // D z = y
        for (int k = K - 2; k >= 0; --k) x[k] -= ll[k + 1] * x[k + 1];  // L^T x = z
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += x[k] * x[k];
        s = 1.0 / sqrt(s);
        for (int k = 0; k < K; ++k) x[k] *= s;
    }
    // sign from psi_0(0) = sum x_k sqrt((4k+1)/2) P_2k(0), P_2k(0) = -P_{2k-2}(0) (2k-1)/(2k)
    double p0 = 1.0, v0 = 0.0;
    for (int k = 0; k < K; ++k) {
        if (k > 0) p0 = -p0 * (2.0 * k - 1.0) / (2.0 * k);
        v0 += x[k] * sqrt((4.0 * k + 1.0) / 2.0) * p0;
    }
    const double sgn = v0 < 0.0 ? -1.0 : 1.0;
    for (int k = 0; k < K; ++k) coef[k] = sgn * x[k] * sqrt((4.0 * k + 1.0) / 2.0);
}

__device__ double legendre_pair(int Q, double x, double* pm1) {
    double p0 = 1.0, p1 = x;
    if (Q == 0) { *pm1 = 0.0; return 1.0; }
    for (int n = 1; n < Q; ++n) {
        const double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pm1 = p0;
    return p1;
}

// Non-negative half of the Gauss-Legendre rule of order Q, ascending:
// th[u] (u = 0 .. Qh-1, Qh = ceil(Q/2)), with the pairing multiplicity folded
// into the weight: wm[u] = m * weight (m = 2 for a node > 0, 1 for node 0).
__global__ void k_gauss_half(int Q, double* __restrict__ th, double* __restrict__ wm) {
    const int Qh = (Q + 1) / 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;   // i-th largest root
    if (i >= Qh) return;
    double x;
    if ((Q & 1) && i == Qh - 1) {
        x = 0.0;
    } else {
        x = cospi((i + 0.75) / (Q + 0.5));
        for (int it = 0; it < 100; ++it) {
            double pm1;
            const double p = legendre_pair(Q, x, &pm1);
            const double dp = Q * (x * p - pm1) / (x * x - 1.0);
            const double dx = p / dp;
            x -= dx;
            if (fabs(dx) <= 1e-16) break;
        }
    }
    double pm1;
    const double p = legendre_pair(Q, x, &pm1);
    const double dp = Q * (x * p - pm1) / (x * x - 1.0);
    const double w = 2.0 / ((1.0 - x * x) * dp * dp);
    const int u = Qh - 1 - i;
    th[u] = x;
    wm[u] = (x > 0.0 ? 2.0 : 1.0) * w;
    (void)p;
}

// Tw[u] = wm[u] * psi_0(th[u]).
__global__ void k_taper(int Qh, const double* __restrict__ th, const double* __restrict__ wm,
                        const double* __restrict__ coef, int K, double* __restrict__ tw) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= Qh) return;
    const double x = th[u];
    double p0 = 1.0, p1 = x, s = coef[0];
    for (int n = 1; n <= 2 * (K - 1); ++n) {
        const double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);
        p0 = p1;
        p1 = p2;
        if (((n + 1) & 1) == 0) s += coef[(n + 1) / 2] * p1;
    }
    tw[u] = wm[u] * s;
}

// A[j][i] = Tw_j Tw_i exp(+j 2 pi w (n - 1)), n - 1 = -r2 / (1 + n).
__global__ void k_screen(int Qh, const double* __restrict__ th, const double* __restrict__ tw,
                         double half, double w, double2* __restrict__ A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= Qh) return;
    const double r2 = (half * half) * (th[i] * th[i] + th[j] * th[j]);
    const double n = sqrt(1.0 - r2);
    const double nm1 = -r2 / (1.0 + n);
    double sn, cs;
    sincospi(2.0 * w * nm1, &sn, &cs);
    const double amp = tw[j] * tw[i];
    A[(int64_t)j * Qh + i] = make_double2(amp * cs, amp * sn);
}

// C[f][u] = cos(pi f th[u] / beta) for f = fmin + fi.
__global__ void k_cosmat(int F, int fmin, int Qh, int beta, const double* __restrict__ th,
                         double* __restrict__ C) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int fi = blockIdx.y;
    if (u >= Qh) return;
    C[(int64_t)fi * Qh + u] = cospi((double)(fmin + fi) * th[u] / (double)beta);
}

// out[m][n] = sum_k X[m][k] * R[n][k]   (X complex M x K, R real N x K)
// written to out[m * ldo + n] (or transposed: out[n * ldo + m]).
template <bool kTransOut>
__global__ void k_gemm_cr(int M, int N, int K, const double2* __restrict__ X,
                          const double* __restrict__ R, double2* __restrict__ out, int ldo) {
    __shared__ double2 sX[32][17];
    __shared__ double sR[32][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads
    const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
    double2 acc[2][2] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 32 * 16; e += 256) {
            const int r = e >> 4, kk = e & 15;
            const int gk = k0 + kk;
            sX[r][kk] = (m0 + r < M && gk < K) ? X[(int64_t)(m0 + r) * K + gk] : make_double2(0, 0);
            sR[r][kk] = (n0 + r < N && gk < K) ? R[(int64_t)(n0 + r) * K + gk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const double2 x0 = sX[ty][kk], x1 = sX[ty + 16][kk];
            const double r0 = sR[tx][kk], r1 = sR[tx + 16][kk];
            acc[0][0].x += x0.x * r0; acc[0][0].y += x0.y * r0;
            acc[0][1].x += x0.x * r1; acc[0][1].y += x0.y * r1;
            acc[1][0].x += x1.x * r0; acc[1][0].y += x1.y * r0;
            acc[1][1].x += x1.x * r1; acc[1][1].y += x1.y * r1;
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int m = m0 + ty + 16 * a, n = n0 + tx + 16 * b;
            if (m < M && n < N) {
                if (kTransOut) out[(int64_t)n * ldo + m] = acc[a][b];
                else out[(int64_t)m * ldo + n] = acc[a][b];
            }
        }
}

// out[m][n] = sum_k R[m][k] * X[n][k]   (R real M x K, X complex N x K)
__global__ void k_gemm_rc(int M, int N, int K, const double* __restrict__ R,
                          const double2* __restrict__ X, double2* __restrict__ out) {
    __shared__ double sR[32][17];
    __shared__ double2 sX[32][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
    double2 acc[2][2] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 32 * 16; e += 256) {
            const int r = e >> 4, kk = e & 15;
            const int gk = k0 + kk;
            sR[r][kk] = (m0 + r < M && gk < K) ? R[(int64_t)(m0 + r) * K + gk] : 0.0;
            sX[r][kk] = (n0 + r < N && gk < K) ? X[(int64_t)(n0 + r) * K + gk] : make_double2(0, 0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const double r0 = sR[ty][kk], r1 = sR[ty + 16][kk];
            const double2 x0 = sX[tx][kk], x1 = sX[tx + 16][kk];
            acc[0][0].x += r0 * x0.x; acc[0][0].y += r0 * x0.y;
            acc[0][1].x += r0 * x1.x; acc[0][1].y += r0 * x1.y;
            acc[1][0].x += r1 * x0.x; acc[1][0].y += r1 * x0.y;
            acc[1][1].x += r1 * x1.x; acc[1][1].y += r1 * x1.y;
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int m = m0 + ty + 16 * a, n = n0 + tx + 16 * b;
            if (m < M && n < N) out[(int64_t)m * N + n] = acc[a][b];
        }
}

// scale = 1 / Re(sum_{tv, tu} Kf0[beta tv - fmin][beta tu - fmin]) over the w = 0 plane.
__global__ void k_scale(const double2* __restrict__ Kf0, int F, int fmin, int beta, int h,
                        double* __restrict__ scale) {
    __shared__ double red[256];
    double s = 0.0;
    const int S = 2 * h + 1;
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
        const int tv = e / S - h, tu = e % S - h;
        s += Kf0[(int64_t)(beta * tv - fmin) * F + (beta * tu - fmin)].x;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int d = blockDim.x / 2; d > 0; d >>= 1) {
        if (threadIdx.x < d) red[threadIdx.x] += red[threadIdx.x + d];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scale[0] = 1.0 / red[0];
        // the largest |K| of all planes: the w = 0, o = 0 centre tap (the
        // integrand there is T(a) T(b) >= 0 with no phase)
        scale[1] = scale[0] * Kf0[(int64_t)(-fmin) * F + (-fmin)].x;
    }
}

// table[((ov' * beta + ou') * S + tv') * S + tu'] = scale * Kf[beta tv - ov - fmin][beta tu - ou - fmin]
// Scaled FP64 entries -> FP32 table and, optionally, a 16-bit table holding
// round(entry * 2^exp2) (one rounding from FP64, to nearest even).
__global__ void k_slices(const double2* __restrict__ Kf, int F, int fmin, int beta, int S,
                         const double* __restrict__ scale, float2* __restrict__ tab,
                         uint32_t* __restrict__ tab16, int kind16, int exp2) {
    const int64_t n = (int64_t)beta * beta * S * S;
    const double sc = *scale;
    const int h = S / 2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int tu = (int)(e % S) - h;
        const int tv = (int)((e / S) % S) - h;
        const int ou = (int)((e / ((int64_t)S * S)) % beta) - beta / 2;
        const int ov = (int)(e / ((int64_t)S * S * beta)) - beta / 2;
        const double2 k = Kf[(int64_t)(beta * tv - ov - fmin) * F + (beta * tu - ou - fmin)];
        const double re = sc * k.x, im = sc * k.y;
        tab[e] = make_float2((float)re, (float)im);
        if (tab16) {
            const double re2 = scalbn(re, exp2), im2 = scalbn(im, exp2);
            uint16_t lo, hi;
            if (kind16 == GW_BF16X2) {
                const __nv_bfloat16 a = __double2bfloat16(re2), b = __double2bfloat16(im2);
                memcpy(&lo, &a, 2);
                memcpy(&hi, &b, 2);
            } else {
                const __half a = __double2half(re2), b = __double2half(im2);
                memcpy(&lo, &a, 2);
                memcpy(&hi, &b, 2);
            }
            tab16[e] = (uint32_t)lo | ((uint32_t)hi << 16);
        }
    }
}

// One-dimensional w = 0 kernel C(f) = sum_u Tw[u] cos(pi f th[u] / beta).
__global__ void k_c1(int F, int fmin, int beta, int Qh, const double* __restrict__ th,
                     const double* __restrict__ tw, double* __restrict__ C1) {
    const int fi = blockIdx.x * blockDim.x + threadIdx.x;
    if (fi >= F) return;
    double s = 0.0;
    for (int u = 0; u < Qh; ++u) s += tw[u] * cospi((double)(fmin + fi) * th[u] / (double)beta);
    C1[fi] = s;
}

// h(l_i) = 1 / (chat(l_i) sinc_beta(l_i)), l_i = (i - N/2) / N,
// chat(l) = (1/beta) sum_f Cn(f) cos(2 pi f l / beta), Cn = C1 / sum_t C1(beta t).
__global__ void k_corrector(int N, int F, int fmin, int beta, int h0,
                            const double* __restrict__ C1, double* __restrict__ hd,
                            float* __restrict__ hf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double norm = 0.0;
    for (int t = -h0; t <= h0; ++t) norm += C1[beta * t - fmin];
    const double l = (double)(i - N / 2) / (double)N;
    double chat = 0.0;
    for (int fi = 0; fi < F; ++fi)
        chat += C1[fi] * cospi(2.0 * (double)(fmin + fi) * l / (double)beta);
    chat = chat / norm / (double)beta;
    const double x = l / (double)beta;
    const double sinc = (x == 0.0) ? 1.0 : sinpi(x) / (M_PI * x);
    const double hv = 1.0 / (chat * sinc);
    hd[i] = hv;
    hf[i] = (float)hv;
}

}  // namespace

cudaError_t build_tables(const TableBuild& tb, float2* d_table, uint32_t* d_table16, int kind16,
                         double* d_h, float* d_hf, double* h_scale, int* h_exp2, double* d_c1,
                         cudaStream_t s) {
    const double c = M_PI * tb.smin / 2.0;
    const int K = (int)std::ceil(0.5 * c) + 40;
    if (K > kMaxTerms) return cudaErrorInvalidValue;
    const int beta = tb.beta;
    // largest per-plane sizes
    int Qmax = 0, Fmax = 0;
    for (int p = 0; p < tb.P; ++p) {
        Qmax = std::max(Qmax, quad_nodes(tb.field, tb.wplane[p], tb.support[p], tb.smin));
        Fmax = std::max(Fmax, beta * tb.support[p]);
    }
    const int Qhmax = (Qmax + 1) / 2;
    double *coef = nullptr, *chi = nullptr, *th = nullptr, *wm = nullptr, *tw = nullptr;
    double *Cm = nullptr, *scale = nullptr, *C1 = nullptr;
    double2 *A = nullptr, *Bt = nullptr, *Kf = nullptr, *Kf0 = nullptr;
    int exp2 = 0;   // storage exponent of the 16-bit table
    cudaError_t err = cudaSuccess;
#define GW_TRY(x) do { err = (x); if (err != cudaSuccess) goto done; } while (0)
    GW_TRY(dev_alloc((void**)&coef, sizeof(double) * K));
    GW_TRY(dev_alloc((void**)&chi, sizeof(double)));
    GW_TRY(dev_alloc((void**)&th, sizeof(double) * Qhmax));
    GW_TRY(dev_alloc((void**)&wm, sizeof(double) * Qhmax));
    GW_TRY(dev_alloc((void**)&tw, sizeof(double) * Qhmax));
    GW_TRY(dev_alloc((void**)&Cm, sizeof(double) * (size_t)Fmax * Qhmax));
    GW_TRY(dev_alloc((void**)&A, sizeof(double2) * (size_t)Qhmax * Qhmax));
    GW_TRY(dev_alloc((void**)&Bt, sizeof(double2) * (size_t)Fmax * Qhmax));
    GW_TRY(dev_alloc((void**)&Kf, sizeof(double2) * (size_t)Fmax * Fmax));
    GW_TRY(dev_alloc((void**)&Kf0, sizeof(double2) * (size_t)(beta * tb.support[0]) * (beta * tb.support[0])));
    GW_TRY(dev_alloc((void**)&scale, 2 * sizeof(double)));
    GW_TRY(dev_alloc((void**)&C1, sizeof(double) * (size_t)beta * tb.support[0]));

    k_pswf<<<1, 1, 0, s>>>(c, K, coef, chi);
    note_launch();
    // plane 0 first (it fixes the scale), then all planes
    for (int pass = 0; pass < 2; ++pass) {
        for (int p = (pass == 0 ? 0 : 0); p < (pass == 0 ? 1 : tb.P); ++p) {
            const int S = tb.support[p];
            const int h = S / 2;
            const int F = beta * S;
            const int fmin = -beta * h - beta / 2 + 1;
            const int Q = quad_nodes(tb.field, tb.wplane[p], S, tb.smin);
            const int Qh = (Q + 1) / 2;
            k_gauss_half<<<(Qh + 127) / 128, 128, 0, s>>>(Q, th, wm);
            k_taper<<<(Qh + 127) / 128, 128, 0, s>>>(Qh, th, wm, coef, K, tw);
            k_screen<<<dim3((Qh + 127) / 128, Qh), 128, 0, s>>>(Qh, th, tw, 0.5 * tb.field,
                                                                tb.wplane[p], A);
            k_cosmat<<<dim3((Qh + 127) / 128, F), 128, 0, s>>>(F, fmin, Qh, beta, th, Cm);
            // Bt[f][j] = sum_i A[j][i] C[f][i]
            k_gemm_cr<true><<<dim3((F + 31) / 32, (Qh + 31) / 32), 256, 0, s>>>(Qh, F, Qh, A, Cm, Bt, Qh);
            // Kf[fv][fu] = sum_j C[fv][j] Bt[fu][j]
            double2* dst = (pass == 0) ? Kf0 : Kf;
            k_gemm_rc<<<dim3((F + 31) / 32, (F + 31) / 32), 256, 0, s>>>(F, F, Qh, Cm, Bt, dst);
            note_launch(6);
            if (pass == 0) {
                k_scale<<<1, 256, 0, s>>>(Kf0, F, fmin, beta, h, scale);
                // corrector from the same w = 0 nodes
                k_c1<<<(F + 127) / 128, 128, 0, s>>>(F, fmin, beta, Qh, th, tw, C1);
                k_corrector<<<(tb.N + 127) / 128, 128, 0, s>>>(tb.N, F, fmin, beta, h, C1, d_h, d_hf);
                note_launch(3);
                if (d_c1)   // the 1-D w = 0 kernel on the fine offsets, kept for hybrid gridding
                    GW_TRY(cudaMemcpyAsync(d_c1, C1, sizeof(double) * F, cudaMemcpyDeviceToDevice, s));
                if (d_table16 && kind16 == GW_F16X2) {
                    // storage exponent from the largest entry: peak * 2^exp2 in [2^14, 2^15)
                    double sp[2];
                    GW_TRY(cudaMemcpyAsync(sp, scale, sizeof sp, cudaMemcpyDeviceToHost, s));
                    GW_TRY(cudaStreamSynchronize(s));
                    int e2 = 0;
                    std::frexp(sp[1], &e2);      // peak = m 2^e2, m in [0.5, 1)
                    exp2 = 15 - e2;
                }
            } else {
                const int64_t n = (int64_t)beta * beta * S * S;
                int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
                k_slices<<<blocks, 256, 0, s>>>(Kf, F, fmin, beta, S, scale, d_table + tb.plane_off[p],
                                                d_table16 ? d_table16 + tb.plane_off[p] : nullptr,
                                                kind16, exp2);
                note_launch();
            }
            GW_TRY(cudaGetLastError());
        }
    }
    GW_TRY(cudaMemcpyAsync(h_scale, scale, sizeof(double), cudaMemcpyDeviceToHost, s));
    GW_TRY(cudaStreamSynchronize(s));
    *h_exp2 = exp2;
done:
#undef GW_TRY
    dev_free(coef); dev_free(chi); dev_free(th); dev_free(wm); dev_free(tw); dev_free(Cm);
    dev_free(A); dev_free(Bt); dev_free(Kf); dev_free(Kf0); dev_free(scale); dev_free(C1);
    return err;
}

namespace {

// Z table of the hybrid pruner: psi_0(c_z, x) at x = (t - o/beta) 2/sz for
// even o in [-beta/2, beta/2) and |t| <= hz, normalised by the sum of its
// zero-offset taps (psi at x = 2t/sz).
__global__ void k_prune_points(int beta, int sz, double* __restrict__ x) {
    const int hz = (sz - 1) / 2, no = beta / 2;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < no * sz) {
        const int row = e / sz, t = e % sz - hz;
        const int o = 2 * row - beta / 2;
        const double v = (t - (double)o / beta) * 2.0 / sz;
        x[e] = fmin(1.0, fmax(-1.0, v));
    } else if (e < no * sz + sz) {
        const int t = e - no * sz - hz;
        x[e] = t * 2.0 / sz;
    }
}

__global__ void k_prune_finish(int beta, int sz, int N, const double* __restrict__ psi,
                               float* __restrict__ z, double* __restrict__ hd,
                               float* __restrict__ hf) {
    const int hz = (sz - 1) / 2, no = beta / 2;
    double norm = 0.0;
    for (int t = 0; t < sz; ++t) norm += psi[no * sz + t];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < no * sz) z[i] = (float)(psi[i] / norm);
    if (i >= N) return;
    // realised transform of Z averaged over the beta/2 offsets, and the
    // nearest-neighbour factor of the beta-fine v rows
    const double x = (double)(i - N / 2) / (double)N;
    double zh = 0.0;
    for (int e = 0; e < no * sz; ++e) {
        const int row = e / sz, t = e % sz - hz;
        const double d = t - (double)(2 * row - beta / 2) / beta;
        zh += psi[e] / norm * cospi(d * x);
    }
    zh *= 2.0 / beta;
    const double a = x / beta;
    const double sinc = (a == 0.0) ? 1.0 : sinpi(a) / (M_PI * a);
    const double hv = 1.0 / (zh * sinc);
    hd[i] = hv;
    hf[i] = (float)hv;
}

}  // namespace

cudaError_t build_prune(int sz, int beta, int N, float* d_z, double* d_hpr, float* d_hprf,
                        cudaStream_t s) {
    const double c = M_PI * sz / 2.0;
    const int K = (int)std::ceil(0.5 * c) + 40;
    if (K > kMaxTerms) return cudaErrorInvalidValue;
    const int np = (beta / 2) * sz + sz;
    double *coef = nullptr, *chi = nullptr, *x = nullptr, *ones = nullptr, *psi = nullptr;
    cudaError_t err = cudaSuccess;
#define GW_TRY(x_) do { err = (x_); if (err != cudaSuccess) goto done; } while (0)
    GW_TRY(dev_alloc((void**)&coef, sizeof(double) * K));
    GW_TRY(dev_alloc((void**)&chi, sizeof(double)));
    GW_TRY(dev_alloc((void**)&x, sizeof(double) * np));
    GW_TRY(dev_alloc((void**)&ones, sizeof(double) * np));
    GW_TRY(dev_alloc((void**)&psi, sizeof(double) * np));
    {
        std::vector<double> h1(np, 1.0);
        GW_TRY(cudaMemcpyAsync(ones, h1.data(), sizeof(double) * np, cudaMemcpyHostToDevice, s));
        k_pswf<<<1, 1, 0, s>>>(c, K, coef, chi);
        k_prune_points<<<(np + 127) / 128, 128, 0, s>>>(beta, sz, x);
        k_taper<<<(np + 127) / 128, 128, 0, s>>>(np, x, ones, coef, K, psi);
        const int nf = std::max(N, (beta / 2) * sz);
        k_prune_finish<<<(nf + 127) / 128, 128, 0, s>>>(beta, sz, N, psi, d_z, d_hpr, d_hprf);
        note_launch(4);
        GW_TRY(cudaGetLastError());
        GW_TRY(cudaStreamSynchronize(s));
    }
done:
#undef GW_TRY
    dev_free(coef); dev_free(chi); dev_free(x); dev_free(ones); dev_free(psi);
    return err;
}

}  // namespace gw
