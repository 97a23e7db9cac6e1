// Kernel table of the vdW-DF nonlocal correlation, built on the device once
// per process and device, then kept resident.
//
//  phi(d1, d2): the vdW kernel cited at Eq. 2 (Dion et al. 2004, published
//    double-integral form) by a tensor-product quadrature in (a, b):
//      phi = sum_ij K_ij T(nu1(a_i), nu1(a_j), nu2(a_i), nu2(a_j))
//      K_ij = (2/pi^2) w_i w_j a_i^2 a_j^2 W(a_i, a_j)
//      W(a,b) = 2 [j0(a) f(b) + j0(b) f(a) - 3 f(a) f(b)],  f(x) = (sin x - x cos x)/x^3
//      T(w,x,y,z) = 1/2 [1/(w+x) + 1/(y+z)] [1/((w+y)(x+z)) + 1/((w+z)(y+x))]
//      nu_i(y) = y^2 / (2 h(y/d_i)),  h(t) = 1 - exp(-4 pi t^2 / 9)
//    Nodes: a = tan(t), t Gauss-Legendre (256 points) on [0, atan(64)].
//  phi_ab(r_i) = phi(q_a r_i, q_b r_i), r_i = i * 100/1024 bohr, i = 0..1024.
//  phi_ab(k_j) = 4 pi int r^2 phi_ab(r) j0(k_j r) dr (composite Simpson),
//    k_j = j * 2 pi / 100 bohr, j = 0..1023 (Sec. 2: the M x M radial
//    functions on a discrete k-grid).
//  Interpolation in k (Sec. 3, procedure step 3a): per interval a cubic in
//    t = k/dk - j, from a natural cubic spline (default) or linear; stored
//    [interval][pair] so that the rows of a |k| range are one contiguous block.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>
#include <chrono>

#include "common.cuh"
#include "table.h"

namespace vdwgb {

static const int NA = 256;          // quadrature nodes per axis
static const double AMAX = 64.0;    // upper end of the a-range
static const int NP_BLK = 16;       // (d1, d2) points per block in k_phi

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n.
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static double j0_host(double x) {
    if (std::fabs(x) < 1e-2) {
        double x2 = x * x;
        return 1.0 - x2 / 6.0 + x2 * x2 / 120.0 - x2 * x2 * x2 / 5040.0;
    }
    return std::sin(x) / x;
}

// f(x) = (sin x - x cos x) / x^3, with its series below 0.1
static double f_host(double x) {
    if (std::fabs(x) < 0.1) {
        double x2 = x * x;
        return 1.0 / 3.0 - x2 / 30.0 + x2 * x2 / 840.0 - x2 * x2 * x2 / 45360.0 +
               x2 * x2 * x2 * x2 / 3991680.0 - x2 * x2 * x2 * x2 * x2 / 518918400.0;
    }
    return (std::sin(x) - x * std::cos(x)) / (x * x * x);
}

void host_qmesh(QMeshDev &q) {
    const double qmin = 1e-5, qcut = 5.0, lam = 1.17;
    const int M = NQ;
    for (int a = 0; a < M; ++a)
        q.q[a] = qmin + (qcut - qmin) * (std::pow(lam, a) - 1.0) / (std::pow(lam, M - 1) - 1.0);
    for (int a = 0; a < M - 1; ++a) {
        q.h[a] = q.q[a + 1] - q.q[a];
        q.invh[a] = 1.0 / q.h[a];
    }
    q.h[M - 1] = q.h[M - 2];
    q.invh[M - 1] = q.invh[M - 2];
    // natural cubic splines through p_a(q_i) = delta_ai: y''_0 = y''_{M-1} = 0,
    // h_{i-1} y''_{i-1} + 2 (h_{i-1} + h_i) y''_i + h_i y''_{i+1} = 6 (dy_i/h_i - dy_{i-1}/h_{i-1})
    std::memset(q.d2, 0, sizeof(q.d2));
    const int n = M - 2;
    for (int a = 0; a < M; ++a) {
        std::vector<double> lo(n), di(n), up(n), rhs(n);
        for (int i = 1; i < M - 1; ++i) {
            const int r = i - 1;
            const double hm = q.h[i - 1], hp = q.h[i];
            lo[r] = hm;
            di[r] = 2.0 * (hm + hp);
            up[r] = hp;
            const double yp = (i + 1 == a), y0 = (i == a), ym = (i - 1 == a);
            rhs[r] = 6.0 * ((yp - y0) / hp - (y0 - ym) / hm);
        }
        // Thomas algorithm
        for (int r = 1; r < n; ++r) {
            const double m = lo[r] / di[r - 1];
            di[r] -= m * up[r - 1];
            rhs[r] -= m * rhs[r - 1];
        }
        std::vector<double> y(n);
        y[n - 1] = rhs[n - 1] / di[n - 1];
        for (int r = n - 2; r >= 0; --r) y[r] = (rhs[r] - up[r] * y[r + 1]) / di[r];
        for (int i = 1; i < M - 1; ++i) q.d2[i * NQ + a] = y[i - 1];
    }
    q.q_min = qmin;
    q.q_cut = qcut;
    q.n_min = 1e-12;
}

// ---------------------------------------------------------------------------
// device kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ double nu_of(double a, double d) {
    if (d == 0.0) return 0.5 * a * a;
    const double t = a / d;
    const double h = -expm1(-(4.0 * 3.14159265358979323846 / 9.0) * t * t);
    return 0.5 * a * a / h;
}

// phi for npts points; each block handles NP_BLK points, thread i = row i.
__global__ void __launch_bounds__(NA) k_phi(int npts, const double *__restrict__ d1, const double *__restrict__ d2,
                                            const double *__restrict__ a, const double *__restrict__ K,
                                            double *__restrict__ out) {
    extern __shared__ double phi_smem[];
    double (*nu1)[NA] = reinterpret_cast<double (*)[NA]>(phi_smem);
    double (*nu2)[NA] = reinterpret_cast<double (*)[NA]>(phi_smem + NP_BLK * NA);
    __shared__ double part[NA / 32][NP_BLK];
    const int p0 = blockIdx.x * NP_BLK;
    const int i = threadIdx.x;
    const double ai = a[i];
    for (int p = 0; p < NP_BLK; ++p) {
        const int gp = min(p0 + p, npts - 1);
        nu1[p][i] = nu_of(ai, d1[gp]);
        nu2[p][i] = nu_of(ai, d2[gp]);
    }
    __syncthreads();
    double w[NP_BLK], y[NP_BLK], acc[NP_BLK];
#pragma unroll
    for (int p = 0; p < NP_BLK; ++p) {
        w[p] = nu1[p][i];
        y[p] = nu2[p][i];
        acc[p] = 0.0;
    }
    for (int j = 0; j < NA; ++j) {
        const double kij = K[(size_t)j * NA + i];   // K symmetric
#pragma unroll
        for (int p = 0; p < NP_BLK; ++p) {
            const double x = nu1[p][j], z = nu2[p][j];
            const double s1 = w[p] + x, s2 = y[p] + z;
            const double s3 = (w[p] + y[p]) * (x + z);
            const double s4 = (w[p] + z) * (y[p] + x);
            // T = 1/2 (1/s1 + 1/s2)(1/s3 + 1/s4)
            const double T = 0.5 * (s1 + s2) * (s3 + s4) / (s1 * s2 * s3 * s4);
            acc[p] += kij * T;
        }
    }
#pragma unroll
    for (int p = 0; p < NP_BLK; ++p) {
        double v = acc[p];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((i & 31) == 0) part[i >> 5][p] = v;
    }
    __syncthreads();
    if (i < NP_BLK && p0 + i < npts) {
        double s = 0.0;
        for (int wv = 0; wv < NA / 32; ++wv) s += part[wv][i];
        out[p0 + i] = s;
    }
}

// g[pair][i] = 4 pi w_i r_i phi_ab(r_i) (Simpson weight w_i); k = 0 row uses r_i^2.
// phik[pair][j] = (1/k_j) sum_i g sin(k_j r_i) for j > 0, sum_i 4 pi w_i r_i^2 phi for j = 0.
// k_j r_i = 2 pi (i j mod NR) / NR.
__global__ void k_ktransform(const double *__restrict__ phir, const double *__restrict__ sintab,
                             double *__restrict__ phik) {
    const int pair = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= NK) return;
    const double dr = RMAX / NR;
    const double dk = 2.0 * 3.14159265358979323846 / RMAX;
    const double *f = phir + (size_t)pair * (NR + 1);
    double s = 0.0;
    if (j == 0) {
        for (int i = 0; i <= NR; ++i) {
            const double wi = (i == 0 || i == NR) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
            const double r = i * dr;
            s += wi * r * r * f[i];
        }
        s *= 4.0 * 3.14159265358979323846 * dr / 3.0;
    } else {
        for (int i = 1; i <= NR; ++i) {
            const double wi = (i == NR) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
            const double r = i * dr;
            s += wi * r * f[i] * sintab[(i * j) & (NR - 1)];
        }
        s *= 4.0 * 3.14159265358979323846 * dr / 3.0 / (j * dk);
    }
    phik[(size_t)pair * NK + j] = s;
}

// Natural cubic spline in k (uniform spacing dk) per pair, then the interval
// polynomials c0 + c1 t + c2 t^2 + c3 t^3, t in [0, 1).
__global__ void k_kspline(const double *__restrict__ phik, double *__restrict__ scratch,
                          dvec4 *__restrict__ cub64, float4 *__restrict__ cub32,
                          dvec4 *__restrict__ lin64, float4 *__restrict__ lin32) {
    const int pair = blockIdx.x * blockDim.x + threadIdx.x;
    if (pair >= NPAIR) return;
    const double dk = 2.0 * 3.14159265358979323846 / RMAX;
    const double *y = phik + (size_t)pair * NK;
    double *cp = scratch + (size_t)pair * 2 * NK;   // modified super-diagonal
    double *y2 = cp + NK;                           // rhs, then y''
    // unknowns y''_1 .. y''_{NK-2}: dk y''_{i-1} + 4 dk y''_i + dk y''_{i+1} = 6 (y_{i+1} - 2 y_i + y_{i-1}) / dk
    const int n = NK - 2;
    double dprev = 0.0;
    for (int r = 0; r < n; ++r) {
        const int i = r + 1;
        const double rhs = 6.0 * (y[i + 1] - 2.0 * y[i] + y[i - 1]) / dk;
        const double diag = 4.0 * dk - (r > 0 ? dk * cp[r - 1] : 0.0);
        cp[r] = dk / diag;
        y2[r] = (rhs - (r > 0 ? dk * dprev : 0.0)) / diag;
        dprev = y2[r];
    }
    for (int r = n - 2; r >= 0; --r) y2[r] -= cp[r] * y2[r + 1];
    // y''_i = y2[i - 1] for 1 <= i <= NK-2, zero at both ends
    const double h26 = dk * dk / 6.0;
    for (int j = 0; j < NK - 1; ++j) {
        const double s0 = (j >= 1 && j <= NK - 2) ? y2[j - 1] : 0.0;
        const double s1 = (j + 1 >= 1 && j + 1 <= NK - 2) ? y2[j] : 0.0;
        const double c0 = y[j];
        const double c1 = (y[j + 1] - y[j]) - h26 * (2.0 * s0 + s1);
        const double c2 = 3.0 * h26 * s0;
        const double c3 = h26 * (s1 - s0);
        const size_t o = (size_t)j * NPAIR + pair;     // [interval][pair]
        cub64[o] = make_dvec4(c0, c1, c2, c3);
        lin64[o] = make_dvec4(y[j], y[j + 1] - y[j], 0.0, 0.0);
        // FP32: pairs 2m, 2m + 1 interleaved as {c0, c0', c1, c1'} {c2, c2', c3, c3'}
        const size_t f = (size_t)j * NPAIR * 4 + (size_t)(pair >> 1) * 8 + (pair & 1);
        float *c32 = reinterpret_cast<float *>(cub32), *l32 = reinterpret_cast<float *>(lin32);
        c32[f] = (float)c0;
        c32[f + 2] = (float)c1;
        c32[f + 4] = (float)c2;
        c32[f + 6] = (float)c3;
        l32[f] = (float)y[j];
        l32[f + 2] = (float)(y[j + 1] - y[j]);
        l32[f + 4] = 0.f;
        l32[f + 6] = 0.f;
    }
}

// ---------------------------------------------------------------------------
// per-device state
// ---------------------------------------------------------------------------
struct DevTable {
    bool built = false;
    double *a = nullptr, *K = nullptr;
    double *phir = nullptr, *phik = nullptr;
    dvec4 *cub64 = nullptr, *lin64 = nullptr;
    float4 *cub32 = nullptr, *lin32 = nullptr;
    double seconds = 0.0;
};

static std::mutex g_mu;
static DevTable g_tab[64];

static cudaError_t quad_to_device(DevTable &t) {
    std::vector<double> x, w;
    gauss_legendre(NA, x, w);
    const double T = std::atan(AMAX);
    std::vector<double> a(NA), wa(NA), K((size_t)NA * NA);
    for (int i = 0; i < NA; ++i) {
        const double tt = 0.5 * (x[i] + 1.0) * T;
        a[i] = std::tan(tt);
        wa[i] = 0.5 * T * w[i] * (1.0 + a[i] * a[i]);
    }
    std::vector<double> fj(NA), j0v(NA);
    for (int i = 0; i < NA; ++i) {
        fj[i] = f_host(a[i]);
        j0v[i] = j0_host(a[i]);
    }
    for (int i = 0; i < NA; ++i)
        for (int j = 0; j < NA; ++j) {
            const double W = 2.0 * (j0v[i] * fj[j] + j0v[j] * fj[i] - 3.0 * fj[i] * fj[j]);
            K[(size_t)i * NA + j] = (2.0 / (M_PI * M_PI)) * wa[i] * wa[j] * a[i] * a[i] * a[j] * a[j] * W;
        }
    cudaError_t e;
    if ((e = cudaMalloc(&t.a, NA * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&t.K, (size_t)NA * NA * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMemcpy(t.a, a.data(), NA * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    return cudaMemcpy(t.K, K.data(), (size_t)NA * NA * sizeof(double), cudaMemcpyHostToDevice);
}

static cudaError_t phi_device(DevTable &t, int npts, const double *dd1, const double *dd2, double *dout,
                              cudaStream_t st) {
    const int blocks = (npts + NP_BLK - 1) / NP_BLK;
    const size_t sm = 2 * NP_BLK * NA * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute((const void *)k_phi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_phi<<<blocks, NA, sm, st>>>(npts, dd1, dd2, t.a, t.K, dout);
    return cudaGetLastError();
}

static cudaError_t build(int device, DevTable &t) {
    auto t0 = std::chrono::steady_clock::now();
    cudaError_t e;
    if ((e = quad_to_device(t)) != cudaSuccess) return e;
    QMeshDev qm;
    host_qmesh(qm);
    // radial points
    const int npts = NPAIR * (NR + 1);
    std::vector<double> d1(npts), d2(npts);
    {
        int p = 0, k = 0;
        for (int a = 0; a < NQ; ++a)
            for (int b = a; b < NQ; ++b, ++p)
                for (int i = 0; i <= NR; ++i, ++k) {
                    const double r = i * (RMAX / NR);
                    d1[k] = qm.q[a] * r;
                    d2[k] = qm.q[b] * r;
                }
    }
    double *dd1 = nullptr, *dd2 = nullptr, *sintab = nullptr, *scratch = nullptr;
    if ((e = cudaMalloc(&dd1, npts * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&dd2, npts * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&t.phir, npts * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&t.phik, (size_t)NPAIR * NK * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&sintab, NR * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&scratch, (size_t)NPAIR * 2 * NK * sizeof(double))) != cudaSuccess) return e;
    const size_t ncoef = (size_t)NPAIR * (NK - 1);
    if ((e = cudaMalloc(&t.cub64, ncoef * sizeof(dvec4))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&t.lin64, ncoef * sizeof(dvec4))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&t.cub32, ncoef * sizeof(float4))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&t.lin32, ncoef * sizeof(float4))) != cudaSuccess) return e;
    std::vector<double> st(NR);
    for (int m = 0; m < NR; ++m) st[m] = std::sin(2.0 * M_PI * m / NR);
    if ((e = cudaMemcpy(dd1, d1.data(), npts * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(dd2, d2.data(), npts * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(sintab, st.data(), NR * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = phi_device(t, npts, dd1, dd2, t.phir, 0)) != cudaSuccess) return e;
    k_ktransform<<<dim3((NK + 127) / 128, NPAIR), 128>>>(t.phir, sintab, t.phik);
    k_kspline<<<(NPAIR + 63) / 64, 64>>>(t.phik, scratch, t.cub64, t.cub32, t.lin64, t.lin32);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
    cudaFree(dd1);
    cudaFree(dd2);
    cudaFree(sintab);
    cudaFree(scratch);
    t.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    t.built = true;
    (void)device;
    return cudaSuccess;
}

cudaError_t table_get(int device, TableRefs &out) {
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    DevTable &t = g_tab[device];
    int prev = -1;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return e;
    if (!t.built) {
        e = build(device, t);
        if (e != cudaSuccess) {
            if (prev >= 0) cudaSetDevice(prev);
            return e;
        }
    }
    out.phir = t.phir;
    out.phik = t.phik;
    out.cub64 = t.cub64;
    out.lin64 = t.lin64;
    out.cub32 = t.cub32;
    out.lin32 = t.lin32;
    out.seconds = t.seconds;
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return cudaSuccess;
}

// The resident table of `device` if it was already built (never builds or
// allocates).
bool table_peek(int device, TableRefs &out) {
    if (device < 0 || device >= 64) return false;
    std::lock_guard<std::mutex> lk(g_mu);
    const DevTable &t = g_tab[device];
    if (!t.built) return false;
    out.phir = t.phir;
    out.phik = t.phik;
    out.cub64 = t.cub64;
    out.lin64 = t.lin64;
    out.cub32 = t.cub32;
    out.lin32 = t.lin32;
    out.seconds = t.seconds;
    return true;
}

double table_seconds(int device) {
    if (device < 0 || device >= 64) return 0.0;
    std::lock_guard<std::mutex> lk(g_mu);
    return g_tab[device].built ? g_tab[device].seconds : 0.0;
}

// Spline coefficients (the same construction as the resident table's) of a
// caller's k-space table, phik[pair * NK + j] on the host; the four arrays
// are allocated here, on the current device.
cudaError_t table_custom(const double *h_phik, CustomTable &out, cudaStream_t st) {
    out = CustomTable{};
    double *phik = nullptr, *scratch = nullptr;
    const size_t ncoef = (size_t)NPAIR * (NK - 1);
    cudaError_t e = cudaMalloc(&phik, (size_t)NPAIR * NK * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&scratch, (size_t)NPAIR * 2 * NK * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&out.cub64, ncoef * sizeof(dvec4));
    if (e == cudaSuccess) e = cudaMalloc(&out.lin64, ncoef * sizeof(dvec4));
    if (e == cudaSuccess) e = cudaMalloc(&out.cub32, ncoef * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&out.lin32, ncoef * sizeof(float4));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(phik, h_phik, (size_t)NPAIR * NK * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k_kspline<<<(NPAIR + 63) / 64, 64, 0, st>>>(phik, scratch, out.cub64, out.cub32, out.lin64, out.lin32);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(phik);
    cudaFree(scratch);
    if (e != cudaSuccess) table_custom_free(out);
    return e;
}

void table_custom_free(CustomTable &t) {
    cudaFree(t.cub64);
    cudaFree(t.lin64);
    cudaFree(t.cub32);
    cudaFree(t.lin32);
    t = CustomTable{};
}

cudaError_t table_phi(int device, int npts, const double *d1, const double *d2, double *out) {
    TableRefs r;
    cudaError_t e = table_get(device, r);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_mu);
    int prev = -1;
    cudaGetDevice(&prev);
    if ((e = cudaSetDevice(device)) != cudaSuccess) return e;
    double *b = nullptr;
    if ((e = cudaMalloc(&b, 3 * (size_t)npts * sizeof(double))) != cudaSuccess) return e;
    cudaMemcpy(b, d1, npts * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(b + npts, d2, npts * sizeof(double), cudaMemcpyHostToDevice);
    e = phi_device(g_tab[device], npts, b, b + npts, b + 2 * npts, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, b + 2 * npts, npts * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(b);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return e;
}

}  // namespace vdwgb
