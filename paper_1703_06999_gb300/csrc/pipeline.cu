// The hot path of the vdW-DF nonlocal correlation (Roman-Perez--Soler FFT
// method, Sec. 2 and the procedure of Sec. 3):
//   zfwd      q0(n, sigma) with saturation (appendix), helper splines p_a,
//             theta_a = n p_a (Eq. theta), real-to-complex FFT along z
//   yfft      complex FFT along y (forward and inverse)
//   xcontract complex FFT along x, kernel interpolation in |k| and the
//             per-k matrix-vector product F_a(k) = sum_b phi_ab(k) theta_b(k)
//             with the energy increment sum_a theta_a^* F_a (procedure step 3),
//             inverse FFT along x
//   zinv      complex-to-real FFT along z and the potential (Eq. dedn,
//             Eq. dedsigma)
//   efinish   deterministic FP64 reduction of the energy partials (Eq. enlk)
// Every kernel walks a global tile list spanning all systems of a launch.
#include "common.cuh"
#include "pipeline.h"

namespace vdwgb {

__constant__ QMeshDev c_qm;

// ---------------------------------------------------------------------------
// q0(n, sigma) in FP64 (appendix): PW92 correlation, gradient term with Z_ab,
// saturation h_5 with 12 terms, clamp to q_min.
// ---------------------------------------------------------------------------
struct Q0 {
    double q0, dqdn, dqds;
    bool live;
};

__device__ __forceinline__ Q0 q0_point(double n, double s, double Z) {
    Q0 r;
    r.live = n > c_qm.n_min;
    if (!r.live) {
        r.q0 = c_qm.q_min;
        r.dqdn = 0.0;
        r.dqds = 0.0;
        return r;
    }
    s = s > 0.0 ? s : 0.0;
    const double A = 0.031091, a1 = 0.2137;
    const double b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
    const double PI = 3.14159265358979323846;
    const double kF = cbrt(3.0 * PI * PI * n);
    const double rs = cbrt(3.0 / (4.0 * PI * n));
    const double srs = sqrt(rs);
    const double D = 2.0 * A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs);
    const double dD = 2.0 * A * (0.5 * b1 / srs + b2 + 1.5 * b3 * srs + 2.0 * b4 * rs);
    const double L = log1p(1.0 / D);
    const double eps = -2.0 * A * (1.0 + a1 * rs) * L;
    const double deps = -2.0 * A * a1 * L + 2.0 * A * (1.0 + a1 * rs) * dD / (D * D + D);
    const double inv_kn2 = 1.0 / (kF * n * n);
    const double G = -(Z / 36.0) * s * inv_kn2;
    const double qraw = kF - (4.0 * PI / 3.0) * eps + G;
    const double inv_n = 1.0 / n;
    const double dq_dn = kF * inv_n / 3.0 + (4.0 * PI / 9.0) * deps * rs * inv_n - (7.0 / 3.0) * G * inv_n;
    const double dq_ds = -(Z / 36.0) * inv_kn2;
    // saturation h_a(x) = a [1 - exp(-sum_{m=1}^{12} (x/a)^m / m)]
    const double a = c_qm.q_cut;
    const double t = qraw / a;
    double S = 0.0, dS = 0.0, tp = 1.0;
#pragma unroll
    for (int m = 1; m <= 12; ++m) {
        dS += tp;          // t^(m-1)
        tp *= t;
        S += tp / (double)m;
    }
    const double e = exp(-S);
    double q0 = a * (1.0 - e);
    double dh = e * dS;
    if (q0 < c_qm.q_min) {
        r.q0 = c_qm.q_min;
        r.dqdn = 0.0;
        r.dqds = 0.0;
        return r;
    }
    r.q0 = q0;
    r.dqdn = dh * dq_dn;
    r.dqds = dh * dq_ds;
    return r;
}

// Interval j with q_j <= q < q_{j+1} (clamped to 0..NQ-2) and B = (q - q_j)/h_j.
__device__ __forceinline__ int q_interval(double q, const double *qs) {
    int lo = 0, hi = NQ - 2;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (qs[mid] <= q) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// p_a(q) for all a, from interval j and spline coordinate B (A = 1 - B):
// p_a = A [a==j] + B [a==j+1] + ((A^3-A) d2_a[j] + (B^3-B) d2_a[j+1]) h^2/6.
template <typename T>
__device__ __forceinline__ void spline_p(int j, T B, T h, const T *d2s, T *p) {
    const T A = (T)1 - B;
    const T cA = (A * A * A - A) * h * h / (T)6;
    const T cB = (B * B * B - B) * h * h / (T)6;
    const T *dj = d2s + j * NQ;
    const T *dj1 = dj + NQ;
#pragma unroll
    for (int a = 0; a < NQ; ++a) p[a] = cA * dj[a] + cB * dj1[a];
#pragma unroll
    for (int a = 0; a < NQ; ++a) {
        if (a == j) p[a] += A;
        if (a == j + 1) p[a] += B;
    }
}

// dp_a/dq: ([a==j+1] - [a==j]) / h + (-(3A^2-1) d2_a[j] + (3B^2-1) d2_a[j+1]) h / 6.
template <typename T>
__device__ __forceinline__ void spline_dp(int j, T B, T h, const T *d2s, T *dp) {
    const T A = (T)1 - B;
    const T dA = -((T)3 * A * A - (T)1) * h / (T)6;
    const T dB = ((T)3 * B * B - (T)1) * h / (T)6;
    const T ih = (T)1 / h;
    const T *dj = d2s + j * NQ;
    const T *dj1 = dj + NQ;
#pragma unroll
    for (int a = 0; a < NQ; ++a) dp[a] = dA * dj[a] + dB * dj1[a];
#pragma unroll
    for (int a = 0; a < NQ; ++a) {
        if (a == j) dp[a] -= ih;
        if (a == j + 1) dp[a] += ih;
    }
}

// Shared q-mesh tables in precision T.
template <typename T>
struct QShared {
    double q[NQ];
    double invh[NQ];
    T h[NQ];
    T d2[NQ * NQ];
};

template <typename T>
__device__ __forceinline__ void load_qshared(QShared<T> *qs) {
    for (int i = threadIdx.x; i < NQ * NQ; i += blockDim.x) qs->d2[i] = (T)c_qm.d2[i];
    for (int i = threadIdx.x; i < NQ; i += blockDim.x) {
        qs->q[i] = c_qm.q[i];
        qs->invh[i] = c_qm.invh[i];
        qs->h[i] = (T)c_qm.h[i];
    }
}

__device__ __forceinline__ size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// z-forward: theta and the real-to-complex transform along z.
// Two real fields share one complex line: c = theta_{2m} + i theta_{2m+1}.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_zfwd(const SysDev *__restrict__ sys, const int *__restrict__ prefix,
                                              int nsys, int total) {
    extern __shared__ __align__(16) unsigned char smem[];
    QShared<T> *qs = reinterpret_cast<QShared<T> *>(smem);
    unsigned char *base = smem + align_up(sizeof(QShared<T>), 16);
    load_qshared(qs);
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int si = find_sys(prefix, nsys, t);
        const SysDev &S = sys[si];
        const int lt = t - prefix[si];
        const int nz = S.nz, nzh = S.nzh, LZ = S.LZ;
        const int nlines_tot = S.nx * S.ny;
        const int l0 = lt * LZ;
        const int nl = min(LZ, nlines_tot - l0);
        const int L = 10 * nl;              // complex lines in this tile
        cx<T> *tw = reinterpret_cast<cx<T> *>(base);
        cx<T> *bufA = tw + nz;
        cx<T> *bufB = bufA + (size_t)nz * L;
        const cx<T> *twg = reinterpret_cast<const cx<T> *>(S.tw[2]);
        for (int i = threadIdx.x; i < nz; i += blockDim.x) tw[i] = twg[i];
        __syncthreads();   // q tables and twiddles ready
        Rec<T> *rec = reinterpret_cast<Rec<T> *>(S.rec);
        const size_t p0 = (size_t)l0 * nz;
        for (int i = threadIdx.x; i < nl * nz; i += blockDim.x) {
            const int li = i / nz, z = i - li * nz;
            const double n = S.n[p0 + i];
            const double sg = S.sigma[p0 + i];
            const Q0 q = q0_point(n, sg, S.Z);
            Rec<T> r;
            T th[NQ];
            if (q.live) {
                const int j = q_interval(q.q0, qs->q);
                const double Bd = (q.q0 - qs->q[j]) * qs->invh[j];
                const T B = (T)Bd;
                T p[NQ];
                spline_p<T>(j, B, qs->h[j], qs->d2, p);
                const T nn = (T)n;
#pragma unroll
                for (int a = 0; a < NQ; ++a) th[a] = nn * p[a];
                r.B = B;
                r.j = j;
                r.ndqn = (T)(n * q.dqdn);
                r.ndqs = (T)(n * q.dqds);
            } else {
#pragma unroll
                for (int a = 0; a < NQ; ++a) th[a] = (T)0;
                r.B = (T)0;
                r.j = -1;
                r.ndqn = (T)0;
                r.ndqs = (T)0;
            }
            rec[p0 + i] = r;
            cx<T> *dst = bufA + (size_t)z * L + li * 10;
#pragma unroll
            for (int c = 0; c < 10; ++c) dst[c] = cx<T>{th[2 * c], th[2 * c + 1]};
        }
        __syncthreads();
        cx<T> *R = fft_lines<false>(bufA, bufB, S.ax[2], L, L, 1, tw, true);
        // unpack the two real transforms and store the half spectrum
        cx<T> *spec = reinterpret_cast<cx<T> *>(S.spec) + (size_t)l0 * nzh * NQ;
        const int nout = nl * nzh * NQ;
        for (int i = threadIdx.x; i < nout; i += blockDim.x) {
            const int a = i % NQ;
            const int rest = i / NQ;
            const int kz = rest % nzh;
            const int li = rest / nzh;
            const int c = a >> 1;
            const cx<T> zk = R[(size_t)kz * L + li * 10 + c];
            const int km = kz == 0 ? 0 : nz - kz;
            const cx<T> zm = R[(size_t)km * L + li * 10 + c];
            cx<T> X;
            if ((a & 1) == 0) {
                X = {(T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y)};
            } else {
                // (zk - conj(zm)) / (2 i)
                const T dx = zk.x - zm.x, dy = zk.y + zm.y;
                X = {(T)0.5 * dy, (T)-0.5 * dx};
            }
            spec[i] = X;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// y transform of a tile (x, kz0 .. kz0 + W - 1), all 20 fields.
// ---------------------------------------------------------------------------
template <typename T, bool INV>
__global__ void __launch_bounds__(256) k_yfft(const SysDev *__restrict__ sys, const int *__restrict__ prefix,
                                              int nsys, int total) {
    extern __shared__ __align__(16) unsigned char smem[];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int si = find_sys(prefix, nsys, t);
        const SysDev &S = sys[si];
        const int lt = t - prefix[si];
        const int ny = S.ny, nzh = S.nzh, W = S.W;
        const int ncol = (nzh + W - 1) / W;
        const int x = lt / ncol;
        const int kz0 = (lt - x * ncol) * W;
        const int wt = min(W, nzh - kz0);
        const int L = wt * NQ;
        cx<T> *tw = reinterpret_cast<cx<T> *>(smem);
        cx<T> *bufA = tw + ny;
        cx<T> *bufB = bufA + (size_t)ny * L;
        const cx<T> *twg = reinterpret_cast<const cx<T> *>(S.tw[1]);
        for (int i = threadIdx.x; i < ny; i += blockDim.x) tw[i] = twg[i];
        cx<T> *spec = reinterpret_cast<cx<T> *>(S.spec);
        const size_t rowstride = (size_t)nzh * NQ;
        const size_t g0 = ((size_t)x * ny * nzh + kz0) * NQ;
        for (int i = threadIdx.x; i < ny * L; i += blockDim.x) {
            const int y = i / L, e = i - y * L;
            bufA[i] = spec[g0 + y * rowstride + e];
        }
        __syncthreads();
        cx<T> *R = fft_lines<INV>(bufA, bufB, S.ax[1], L, L, 1, tw, true);
        for (int i = threadIdx.x; i < ny * L; i += blockDim.x) {
            const int y = i / L, e = i - y * L;
            spec[g0 + y * rowstride + e] = R[i];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// x transform + kernel contraction + energy + inverse x transform.
// Tile (ky, kz0 .. kz0 + W - 1); after the forward x transform every k-point
// of the tile has its 20 theta_a(k) in shared memory.
// ---------------------------------------------------------------------------
template <typename T>
struct KTab;
template <>
struct KTab<float> {
    using V = float4;
};
template <>
struct KTab<double> {
    using V = dvec4;
};

__device__ __forceinline__ float4 ld_tab(const float4 *p) { return __ldg(p); }
__device__ __forceinline__ dvec4 ld_tab(const dvec4 *p) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return make_dvec4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ int fold(int i, int n) { return i <= (n - 1) / 2 ? i : i - n; }

template <typename T>
__device__ __forceinline__ void contract_point(cx<T> *v, T kabs, const typename KTab<T>::V *__restrict__ tab,
                                               T inv_dk, T weight, double &eacc) {
    cx<T> th[NQ];
#pragma unroll
    for (int a = 0; a < NQ; ++a) th[a] = v[a];
    cx<T> F[NQ];
#pragma unroll
    for (int a = 0; a < NQ; ++a) F[a] = cx<T>{(T)0, (T)0};
    const T xk = kabs * inv_dk;
    int j = (int)xk;                         // kabs >= 0
    if (j < NK - 1) {
        const T tt = xk - (T)j;
        const typename KTab<T>::V *row = tab + j;
        int pidx = 0;
#pragma unroll
        for (int a = 0; a < NQ; ++a) {
#pragma unroll
            for (int b = a; b < NQ; ++b) {
                const typename KTab<T>::V c = ld_tab(row + (size_t)pidx * (NK - 1));
                const T phi = c.x + tt * (c.y + tt * (c.z + tt * c.w));
                F[a].x += phi * th[b].x;
                F[a].y += phi * th[b].y;
                if (b != a) {
                    F[b].x += phi * th[a].x;
                    F[b].y += phi * th[a].y;
                }
                ++pidx;
            }
        }
    }
    T e = (T)0;
#pragma unroll
    for (int a = 0; a < NQ; ++a) e += th[a].x * F[a].x + th[a].y * F[a].y;
    eacc += (double)(weight * e);
#pragma unroll
    for (int a = 0; a < NQ; ++a) v[a] = F[a];
}

template <typename T>
__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) s += red[i];
    }
    __syncthreads();
    return s;
}

template <typename T>
__global__ void __launch_bounds__(256) k_xcontract(const SysDev *__restrict__ sys, const int *__restrict__ prefix,
                                                   int nsys, int total,
                                                   const typename KTab<T>::V *__restrict__ tab) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    const T inv_dk = (T)(RMAX / (2.0 * 3.14159265358979323846));
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int si = find_sys(prefix, nsys, t);
        const SysDev &S = sys[si];
        const int lt = t - prefix[si];
        const int nx = S.nx, ny = S.ny, nz = S.nz, nzh = S.nzh, W = S.W;
        const int ncol = (nzh + W - 1) / W;
        const int ky = lt / ncol;
        const int kz0 = (lt - ky * ncol) * W;
        const int wt = min(W, nzh - kz0);
        const int L = wt * NQ;
        cx<T> *tw = reinterpret_cast<cx<T> *>(smem);
        cx<T> *bufA = tw + nx;
        cx<T> *bufB = bufA + (size_t)nx * L;
        const cx<T> *twg = reinterpret_cast<const cx<T> *>(S.tw[0]);
        for (int i = threadIdx.x; i < nx; i += blockDim.x) tw[i] = twg[i];
        cx<T> *spec = reinterpret_cast<cx<T> *>(S.spec);
        const size_t rowstride = (size_t)ny * nzh * NQ;
        const size_t g0 = ((size_t)ky * nzh + kz0) * NQ;
        for (int i = threadIdx.x; i < nx * L; i += blockDim.x) {
            const int x = i / L, e = i - x * L;
            bufA[i] = spec[g0 + x * rowstride + e];
        }
        __syncthreads();
        cx<T> *R = fft_lines<false>(bufA, bufB, S.ax[0], L, L, 1, tw, true);
        cx<T> *O = R == bufA ? bufB : bufA;
        // contraction, one thread per k-point
        double eacc = 0.0;
        const int my = fold(ky, ny);
        const bool nyq_y = (ny % 2 == 0) && (ky == ny / 2);
        const T g00 = (T)S.g[0], g11 = (T)S.g[1], g22 = (T)S.g[2];
        const T g01 = (T)S.g[3], g02 = (T)S.g[4], g12 = (T)S.g[5];
        for (int i = threadIdx.x; i < nx * wt; i += blockDim.x) {
            const int x = i / wt, w = i - x * wt;
            const int kz = kz0 + w;
            const int mx = fold(x, nx);
            const bool nyq_x = (nx % 2 == 0) && (x == nx / 2);
            const bool nyq_z = (nz % 2 == 0) && (kz == nz / 2);
            const int mz = nyq_z ? -kz : kz;
            const T fx = (T)mx, fy = (T)my, fz = (T)mz;
            const T cxv = nyq_x ? (T)0 : fx, cyv = nyq_y ? (T)0 : fy, czv = nyq_z ? (T)0 : fz;
            T k2 = g00 * fx * fx + g11 * fy * fy + g22 * fz * fz +
                   (T)2 * (g01 * cxv * cyv + g02 * cxv * czv + g12 * cyv * czv);
            k2 = k2 > (T)0 ? k2 : (T)0;
            const T kabs = sqrt(k2);
            const T weight = (kz == 0 || nyq_z) ? (T)1 : (T)2;
            contract_point<T>(R + (size_t)x * L + w * NQ, kabs, tab, inv_dk, weight, eacc);
        }
        const double es = block_sum<T>(eacc, red);
        if (threadIdx.x == 0) S.epart[lt] = es;
        __syncthreads();
        cx<T> *R2 = fft_lines<true>(R, O, S.ax[0], L, L, 1, tw, true);
        for (int i = threadIdx.x; i < nx * L; i += blockDim.x) {
            const int x = i / L, e = i - x * L;
            spec[g0 + x * rowstride + e] = R2[i];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// z-inverse: complex-to-real along z, then the potential.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_zinv(const SysDev *__restrict__ sys, const int *__restrict__ prefix,
                                              int nsys, int total) {
    extern __shared__ __align__(16) unsigned char smem[];
    QShared<T> *qs = reinterpret_cast<QShared<T> *>(smem);
    unsigned char *base = smem + align_up(sizeof(QShared<T>), 16);
    load_qshared(qs);
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int si = find_sys(prefix, nsys, t);
        const SysDev &S = sys[si];
        const int lt = t - prefix[si];
        const int nz = S.nz, nzh = S.nzh, LZ = S.LZ;
        const int nlines_tot = S.nx * S.ny;
        const int l0 = lt * LZ;
        const int nl = min(LZ, nlines_tot - l0);
        const int L = 10 * nl;
        cx<T> *tw = reinterpret_cast<cx<T> *>(base);
        cx<T> *bufA = tw + nz;
        cx<T> *bufB = bufA + (size_t)nz * L;
        const cx<T> *twg = reinterpret_cast<const cx<T> *>(S.tw[2]);
        for (int i = threadIdx.x; i < nz; i += blockDim.x) tw[i] = twg[i];
        const cx<T> *spec = reinterpret_cast<const cx<T> *>(S.spec) + (size_t)l0 * nzh * NQ;
        const bool even = (nz % 2) == 0;
        // Z_c[kz] = X_{2c}[kz] + i X_{2c+1}[kz]; Z_c[nz-kz] = conj(X_{2c}) + i conj(X_{2c+1})
        for (int i = threadIdx.x; i < nl * nzh * 10; i += blockDim.x) {
            const int c = i % 10;
            const int rest = i / 10;
            const int kz = rest % nzh;
            const int li = rest / nzh;
            cx<T> a = spec[(size_t)rest * NQ + 2 * c];
            cx<T> b = spec[(size_t)rest * NQ + 2 * c + 1];
            if (kz == 0 || (even && kz == nz / 2)) {
                a.y = (T)0;
                b.y = (T)0;
            }
            bufA[(size_t)kz * L + li * 10 + c] = cx<T>{a.x - b.y, a.y + b.x};
            const int km = nz - kz;
            if (kz > 0 && km >= nzh)
                bufA[(size_t)km * L + li * 10 + c] = cx<T>{a.x + b.y, b.x - a.y};
        }
        __syncthreads();
        cx<T> *R = fft_lines<true>(bufA, bufB, S.ax[2], L, L, 1, tw, true);
        const Rec<T> *rec = reinterpret_cast<const Rec<T> *>(S.rec);
        const size_t p0 = (size_t)l0 * nz;
        const T invN = (T)S.invN;
        for (int i = threadIdx.x; i < nl * nz; i += blockDim.x) {
            const int li = i / nz, z = i - li * nz;
            const Rec<T> r = rec[p0 + i];
            double dn = 0.0, ds = 0.0;
            if (r.j >= 0) {
                T p[NQ], dp[NQ];
                spline_p<T>(r.j, r.B, qs->h[r.j], qs->d2, p);
                spline_dp<T>(r.j, r.B, qs->h[r.j], qs->d2, dp);
                const cx<T> *src = R + (size_t)z * L + li * 10;
                T s0 = (T)0, s1 = (T)0;
#pragma unroll
                for (int c = 0; c < 10; ++c) {
                    const cx<T> v = src[c];
                    s0 += v.x * p[2 * c] + v.y * p[2 * c + 1];
                    s1 += v.x * dp[2 * c] + v.y * dp[2 * c + 1];
                }
                s0 *= invN;
                s1 *= invN;
                dn = (double)(s0 + r.ndqn * s1);
                ds = (double)(r.ndqs * s1);
            }
            S.dedn[p0 + i] = dn;
            S.dedsigma[p0 + i] = ds;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Energy: E = 1/2 (Omega / N^2) sum_k w_k sum_a Re(theta_a^* F_a), partials
// summed in a fixed order with Neumaier compensation (one block per system).
// ---------------------------------------------------------------------------
__global__ void k_efinish(const SysDev *__restrict__ sys, int nsys) {
    __shared__ double ssum[256], scmp[256];
    for (int si = blockIdx.x; si < nsys; si += gridDim.x) {
        const SysDev &S = sys[si];
        const int n = S.tiles[2];
        double s = 0.0, c = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const double v = S.epart[i];
            const double tt = s + v;
            c += fabs(s) >= fabs(v) ? (s - tt) + v : (v - tt) + s;
            s = tt;
        }
        ssum[threadIdx.x] = s;
        scmp[threadIdx.x] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            double S2 = 0.0, C2 = 0.0;
            for (int i = 0; i < (int)blockDim.x; ++i) {
                const double v = ssum[i];
                const double tt = S2 + v;
                C2 += fabs(S2) >= fabs(v) ? (S2 - tt) + v : (v - tt) + S2;
                S2 = tt;
                C2 += scmp[i];
            }
            *S.energy = S.escale * (S2 + C2);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
template <typename T>
size_t smem_z(int nz, int LZ) {
    return ((sizeof(QShared<T>) + 15) / 16) * 16 + sizeof(cx<T>) * ((size_t)nz + 2ull * nz * 10 * LZ);
}
template <typename T>
size_t smem_xy(int n, int W) {
    return sizeof(cx<T>) * ((size_t)n + 2ull * n * NQ * W);
}

size_t stage_smem(int stage, int prec, int n, int tile) {
    const bool f = prec == 1;
    switch (stage) {
        case 0:
        case 3: return f ? smem_z<float>(n, tile) : smem_z<double>(n, tile);
        default: return f ? smem_xy<float>(n, tile) : smem_xy<double>(n, tile);
    }
}

static cudaError_t set_smem(const void *fn, size_t bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
static cudaError_t init_kernels_t(size_t maxsmem) {
    cudaError_t e;
    if ((e = set_smem((const void *)k_zfwd<T>, maxsmem)) != cudaSuccess) return e;
    if ((e = set_smem((const void *)k_yfft<T, false>, maxsmem)) != cudaSuccess) return e;
    if ((e = set_smem((const void *)k_yfft<T, true>, maxsmem)) != cudaSuccess) return e;
    if ((e = set_smem((const void *)k_xcontract<T>, maxsmem - 32 * sizeof(double))) != cudaSuccess) return e;
    if ((e = set_smem((const void *)k_zinv<T>, maxsmem)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t init_kernels(size_t maxsmem) {
    cudaError_t e = init_kernels_t<float>(maxsmem);
    if (e != cudaSuccess) return e;
    return init_kernels_t<double>(maxsmem);
}

template <typename T>
static cudaError_t launch_all_t(const LaunchSet &ls, cudaStream_t st, cudaEvent_t *ev) {
    const typename KTab<T>::V *tab = reinterpret_cast<const typename KTab<T>::V *>(ls.table);
    if (ev) cudaEventRecord(ev[0], st);
    k_zfwd<T><<<ls.grid[0], 256, ls.smem[0], st>>>(ls.sys, ls.prefix[0], ls.nsys, ls.total[0]);
    if (ev) cudaEventRecord(ev[1], st);
    k_yfft<T, false><<<ls.grid[1], 256, ls.smem[1], st>>>(ls.sys, ls.prefix[1], ls.nsys, ls.total[1]);
    if (ev) cudaEventRecord(ev[2], st);
    k_xcontract<T><<<ls.grid[2], 256, ls.smem[2], st>>>(ls.sys, ls.prefix[2], ls.nsys, ls.total[2], tab);
    if (ev) cudaEventRecord(ev[3], st);
    k_yfft<T, true><<<ls.grid[1], 256, ls.smem[1], st>>>(ls.sys, ls.prefix[1], ls.nsys, ls.total[1]);
    if (ev) cudaEventRecord(ev[4], st);
    k_zinv<T><<<ls.grid[3], 256, ls.smem[3], st>>>(ls.sys, ls.prefix[3], ls.nsys, ls.total[3]);
    if (ev) cudaEventRecord(ev[5], st);
    k_efinish<<<ls.nsys < 1024 ? ls.nsys : 1024, 256, 0, st>>>(ls.sys, ls.nsys);
    if (ev) cudaEventRecord(ev[6], st);
    return cudaGetLastError();
}

cudaError_t launch_all(const LaunchSet &ls, int prec, cudaStream_t st, cudaEvent_t *ev) {
    return prec == 1 ? launch_all_t<float>(ls, st, ev) : launch_all_t<double>(ls, st, ev);
}

const char *stage_name(int i) {
    static const char *names[NSTAGE] = {"zfwd", "yfwd", "xcontract", "yinv", "zinv", "efinish"};
    return (i >= 0 && i < NSTAGE) ? names[i] : "";
}


cudaError_t upload_qmesh(const QMeshDev &q) { return cudaMemcpyToSymbol(c_qm, &q, sizeof(QMeshDev)); }

}  // namespace vdwgb
