// Shared device-side definitions of the vdW-DF nonlocal-correlation library:
// complex type, per-system descriptors, shared-memory mixed-radix FFT.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vdwgb {

constexpr int NQ = 20;                    // q-mesh points M (Sec. 2: M = 20)
constexpr int NPAIR = NQ * (NQ + 1) / 2;  // symmetric kernel pairs (a <= b)
constexpr int NR = 1024;                  // radial intervals of the kernel table
constexpr int NK = 1024;                  // k points of the kernel table
constexpr double RMAX = 100.0;            // radial extent of the kernel table (bohr)
constexpr int MAXST = 12;                 // max FFT stages per axis

// Four doubles, 32-byte aligned (interval polynomial of the FP64 kernel table).
struct __align__(32) dvec4 {
    double x, y, z, w;
};
__host__ __device__ __forceinline__ dvec4 make_dvec4(double x, double y, double z, double w) {
    dvec4 v;
    v.x = x;
    v.y = y;
    v.z = z;
    v.w = w;
    return v;
}

template <typename T>
struct __align__(2 * sizeof(T)) cx {
    T x, y;
};

template <typename T>
__device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// Two FP32 values in one 64-bit register pair, and the two-lane FP32 FMA of
// sm_100-family GPUs (d = a * b + c per lane, round to nearest).
__device__ __forceinline__ unsigned long long pack_f2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack_f2(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long fma_f2(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// multiply by -i (forward) or +i (inverse)
template <bool INV, typename T>
__device__ __forceinline__ cx<T> mul_mi(cx<T> a) {
    return INV ? cx<T>{-a.y, a.x} : cx<T>{a.y, -a.x};
}

// One axis of a 3-D transform: length and its radix factorisation.
struct AxisPlan {
    int n;
    int nst;
    int rad[MAXST];
};

// Per-point record kept from the forward pass for the potential pass.
template <typename T>
struct Rec;
template <>
struct __align__(16) Rec<float> {
    float B;       // spline coordinate in the q-interval
    int j;         // q-interval, -1 for points at or below the density cut-off
    float ndqn;    // n dq0/dn
    float ndqs;    // n dq0/dsigma
};
template <>
struct __align__(16) Rec<double> {
    double B;
    double ndqn;
    double ndqs;
    int j;
    int pad;
};

// Device descriptor of one system of a launch (one handle).
struct SysDev {
    int nx, ny, nz, nzh;
    int LZ;          // z-lines per tile of the z-forward pass
    int LZi;         // z-lines per tile of the z-inverse pass
    int Wy, Wx;      // k_z columns per tile of the y and x passes
    int tiles[6];    // tiles of: z-forward, y, x, z-inverse, contraction chunks, kz-planes
    AxisPlan ax[3];  // x, y, z
    const void *tw[3];   // twiddles exp(-2 pi i m / n), m < n, per axis (T complex)
    double g[6];     // reciprocal metric g00 g11 g22 g01 g02 g12 (|k|^2 = m^T g m)
    float gf[6];     // the same in FP32
    double escale;   // 1/2 Omega / N^2
    double invN;     // 1 / N
    double Z;        // Z_ab of the functional
    float zc[2];     // -Z_ab / 36 as an FP32 pair (hi, lo), for the FP32-mixed q0
    float invNf;     // 1 / N in FP32
    int q0in;        // 1: sigma holds q0 (spin-polarised form: q0 formed beforehand) and the
                     // z-inverse pass writes sum_a F_a p_a and n sum_a F_a p'_a as dedn / dedsigma
    const double *n;
    const double *sigma;
    double *dedn;
    double *dedsigma;
    void *spec;      // [nx][ny][nzh][20] complex (T)
    void *rec;       // [nx*ny*nz] Rec<T>
    const unsigned *kidx;   // half-spectrum k-points sorted by kernel-table interval
    const int4 *chunks;     // contraction chunks: {first, count, first interval, intervals}
    double *epart;   // energy partials (per contraction chunk, or per plane and cluster rank)
    int nepart;      // number of energy partials
    // plane kernel (fused y / x transforms and contraction), else zero:
    int fused;       // cluster size C; each CTA owns nx / C x-rows, then ny / C y-rows
    int sx1, sy1;    // N1 of the two-pass splits of the x and y axes
    int sz1;         // FP32: N1 of the in-place split of the z axis (0: none, out-of-place z passes)
    int kstride;     // entries per (kz, rank) list of kord
    int yoff, nyg;   // y positions [yoff, yoff + ny) of a global y axis of length nyg (a slab of
                     // the k-space half of a slab decomposition); 0 and ny otherwise
    const unsigned short *kord;   // per (kz, rank): local k-point indices sorted by table interval
    const void *tmap;    // FP32: two tensor maps of spec (y-pass tile box, x-pass tile box), else null
    int tby, tbx;        // rows per tensor copy of a y / x tile (a divisor of ny / nx, <= 256)
    double *energy;  // output (device)
    int *err;        // device status flag (and detail word) of the device
};

// Bounds checks of the checked build (VDWGB_CHECK_BOUNDS defined): a failed
// check sets status 3 and the source line in the flag's detail word, and the
// caller skips the access or tile; without the define every check is the
// constant true and compiles away.
#ifdef VDWGB_CHECK_BOUNDS
__device__ __forceinline__ bool vdwgb_check(bool ok, int *err, int line) {
    if (!ok) {
        atomicExch(err + 1, line);
        atomicExch(err, 3);
    }
    return ok;
}
#define VDWGB_OK(cond, err) vdwgb::vdwgb_check((cond), (err), __LINE__)
#else
#define VDWGB_OK(cond, err) true
#endif

// Library-wide constants on the device (q-mesh and helper-spline data).
struct QMeshDev {
    double q[NQ];
    double invh[NQ];       // 1 / (q_{j+1} - q_j)
    double h[NQ];
    double d2[NQ * NQ];    // d2[j * NQ + a]: second derivative of p_a at node j
    double q_min, q_cut, n_min;
};

// ---------------------------------------------------------------------------
// Small DFTs (forward: exp(-2 pi i r k / R); INV: conjugate)
// ---------------------------------------------------------------------------
template <bool INV, typename T>
__device__ __forceinline__ void dft2(cx<T> *v) {
    cx<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <bool INV, typename T>
__device__ __forceinline__ void dft4(cx<T> *v) {
    cx<T> t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    cx<T> t2 = cadd(v[1], v[3]), t3 = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
}

template <bool INV, typename T>
__device__ __forceinline__ void dft8(cx<T> *v) {
    cx<T> e[4] = {v[0], v[2], v[4], v[6]};
    cx<T> o[4] = {v[1], v[3], v[5], v[7]};
    dft4<INV>(e);
    dft4<INV>(o);
    const T s = (T)0.70710678118654752440;
    // o[k] *= W8^k, W8 = exp(-+ 2 pi i / 8)
    cx<T> o1 = INV ? cx<T>{s * (o[1].x - o[1].y), s * (o[1].x + o[1].y)}
                   : cx<T>{s * (o[1].x + o[1].y), s * (o[1].y - o[1].x)};
    cx<T> o2 = mul_mi<INV>(o[2]);
    cx<T> o3 = INV ? cx<T>{-s * (o[3].x + o[3].y), s * (o[3].x - o[3].y)}
                   : cx<T>{s * (o[3].y - o[3].x), -s * (o[3].x + o[3].y)};
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
}

template <bool INV, typename T>
__device__ __forceinline__ void dft3(cx<T> *v) {
    const T c = (T)-0.5, s = (T)0.86602540378443864676;   // cos, sin of 2 pi / 3
    cx<T> t1 = cadd(v[1], v[2]);
    cx<T> d = csub(v[1], v[2]);
    cx<T> m = {v[0].x + c * t1.x, v[0].y + c * t1.y};
    // forward: -i s d ; inverse: +i s d
    cx<T> r = INV ? cx<T>{-s * d.y, s * d.x} : cx<T>{s * d.y, -s * d.x};
    v[0] = cadd(v[0], t1);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
}

// Odd prime radix R (5 or 7) by pairing r and R - r:
// y_k = a0 + sum_r s_r cos(2 pi r k/R) -+ i d_r sin(2 pi r k/R), s_r = a_r + a_{R-r}, d_r = a_r - a_{R-r}.
template <int R, bool INV, typename T>
__device__ __forceinline__ void dft_odd(cx<T> *v) {
    constexpr int H = (R - 1) / 2;
    // cos(2 pi m / R), sin(2 pi m / R) for m = 0..R-1
    const double C5[5] = {1.0, 0.30901699437494742410, -0.80901699437494742410,
                          -0.80901699437494742410, 0.30901699437494742410};
    const double S5[5] = {0.0, 0.95105651629515357212, 0.58778525229247312917,
                          -0.58778525229247312917, -0.95105651629515357212};
    const double C7[7] = {1.0, 0.62348980185873353053, -0.22252093395631440429,
                          -0.90096886790241912624, -0.90096886790241912624,
                          -0.22252093395631440429, 0.62348980185873353053};
    const double S7[7] = {0.0, 0.78183148246802980871, 0.97492791218182360702,
                          0.43388373911755812048, -0.43388373911755812048,
                          -0.97492791218182360702, -0.78183148246802980871};
    cx<T> sr[H], dr[H];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
        sr[r - 1] = cadd(v[r], v[R - r]);
        dr[r - 1] = csub(v[r], v[R - r]);
    }
    cx<T> a0 = v[0];
    cx<T> y0 = a0;
#pragma unroll
    for (int r = 0; r < H; ++r) y0 = cadd(y0, sr[r]);
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        cx<T> A = a0, Bv = {0, 0};
#pragma unroll
        for (int r = 1; r <= H; ++r) {
            const int m = (r * k) % R;
            const T c = (T)(R == 5 ? C5[m] : C7[m]);
            const T s = (T)(R == 5 ? S5[m] : S7[m]);
            A.x += c * sr[r - 1].x;
            A.y += c * sr[r - 1].y;
            Bv.x += s * dr[r - 1].x;
            Bv.y += s * dr[r - 1].y;
        }
        // forward: y_k = A - i B, y_{R-k} = A + i B
        cx<T> iB = {-Bv.y, Bv.x};
        if (INV) {
            v[k] = cadd(A, iB);
            v[R - k] = csub(A, iB);
        } else {
            v[k] = csub(A, iB);
            v[R - k] = cadd(A, iB);
        }
    }
    v[0] = y0;
}

template <int R, bool INV, typename T>
__device__ __forceinline__ void dft(cx<T> *v) {
    if constexpr (R == 2) dft2<INV>(v);
    else if constexpr (R == 3) dft3<INV>(v);
    else if constexpr (R == 4) dft4<INV>(v);
    else if constexpr (R == 8) dft8<INV>(v);
    else dft_odd<R, INV>(v);
}

// One Stockham stage (radix R) over `nlines` lines held in shared memory:
// element i of line l sits at buf[i * ld + l] (ld >= nlines).  Thread tid works on line
// tid % nlines and butterflies j = tid / nlines, + jstep, ... (jstep =
// blockDim / nlines; the last blockDim % nlines threads idle), so the loop
// needs no division; q = j / Ns and jm = j % Ns are carried along.
// Ns = product of the radices already applied.
template <int R, bool INV, typename T>
__device__ __forceinline__ void fft_stage(const cx<T> *in, cx<T> *out, int n, int Ns, int ld, int line,
                                          int j0, int jstep, const cx<T> *tw) {
    const int nb = n / R;
    const int tws = n / (Ns * R);
    int q = j0 / Ns;
    int jm = j0 - q * Ns;
    for (int j = j0; j < nb; j += jstep) {
        cx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[(j + r * nb) * ld + line];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                cx<T> w = tw[jm * r * tws];
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft<R, INV>(v);
        const int base = q * Ns * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) out[(base + r * Ns) * ld + line] = v[r];
        jm += jstep;
        while (jm >= Ns) {
            jm -= Ns;
            ++q;
        }
    }
}

// Full 1-D transforms of `nlines` lines (unnormalised), layout [i][ld].
// Ping-pongs between a and b; returns the buffer that holds the result.
// Ends with a barrier.  Lines are taken in groups of at most blockDim.x.
template <bool INV, typename T>
__device__ cx<T> *fft_lines(cx<T> *a, cx<T> *b, const AxisPlan &p, int nlines, int ld, const cx<T> *tw) {
    const int nt = blockDim.x;
    int Ns = 1;
    for (int s = 0; s < p.nst; ++s) {
        const int R = p.rad[s];
        for (int lb = 0; lb < nlines; lb += nt) {
            const int ng = min(nlines - lb, nt);      // lines in this group
            const int jstep = nt / ng;
            const int j0 = threadIdx.x / ng;
            const int line = lb + threadIdx.x - j0 * ng;
            if (j0 < jstep) {
                switch (R) {
                    case 2: fft_stage<2, INV>(a, b, p.n, Ns, ld, line, j0, jstep, tw); break;
                    case 3: fft_stage<3, INV>(a, b, p.n, Ns, ld, line, j0, jstep, tw); break;
                    case 4: fft_stage<4, INV>(a, b, p.n, Ns, ld, line, j0, jstep, tw); break;
                    case 5: fft_stage<5, INV>(a, b, p.n, Ns, ld, line, j0, jstep, tw); break;
                    case 7: fft_stage<7, INV>(a, b, p.n, Ns, ld, line, j0, jstep, tw); break;
                    default: fft_stage<8, INV>(a, b, p.n, Ns, ld, line, j0, jstep, tw); break;
                }
            }
        }
        __syncthreads();
        cx<T> *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// Find the system that owns global tile t (prefix[s] <= t < prefix[s+1]).
__device__ __forceinline__ int find_sys(const int *prefix, int nsys, int t) {
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Tiles are walked in increasing order, so the owning system only moves
// forward: advance from the current owner (usually zero or one step).
__device__ __forceinline__ int advance_sys(const int *prefix, int nsys, int t, int si) {
    if (si < 0) return find_sys(prefix, nsys, t);
    while (si + 1 < nsys && prefix[si + 1] <= t) ++si;
    return si;
}

// Copy a system descriptor into shared memory (all threads of the block).
__device__ __forceinline__ void copy_sys(SysDev *dst, const SysDev *src) {
    const int *s = reinterpret_cast<const int *>(src);
    int *d = reinterpret_cast<int *>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(SysDev) / sizeof(int)); i += blockDim.x) d[i] = s[i];
}

}  // namespace vdwgb
