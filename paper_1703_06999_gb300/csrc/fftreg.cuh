// Register-resident FFT codelets and a two-pass line transform for axis
// lengths known at compile time.
//
// A length N = N1 * N2 transform of many lines held in shared memory (element
// i of line l at buf[i * ld + l]) runs as two passes (Cooley-Tukey, Sec. 3
// uses a library FFT; this is the GB300 replacement):
//   pass A: for each (line, j2): the N1 elements j1 * N2 + j2 are loaded into
//           registers, transformed by a length-N1 codelet, multiplied by the
//           twiddles W_N^(j2 k1) and stored to scratch at (k1 * N2 + j2);
//   pass B: for each (line, k1): the N2 scratch elements k1 * N2 + j2 are
//           transformed by a length-N2 codelet and stored back at k1 + N1 k2.
// Each pass is one barrier; codelet twiddles are compile-time constants.
#pragma once
#include "common.cuh"

namespace vdwgb {

// ---- compile-time cos and sin (Taylor series on an octant) ---------------
constexpr double kPiC = 3.14159265358979323846264338327950288;

constexpr double taylor_sin(double x) {   // |x| <= pi / 4
    double x2 = x * x, term = x, sum = x;
    for (int k = 1; k < 14; ++k) {
        term *= -x2 / (double)((2 * k) * (2 * k + 1));
        sum += term;
    }
    return sum;
}

constexpr double taylor_cos(double x) {   // |x| <= pi / 4
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int k = 1; k < 14; ++k) {
        term *= -x2 / (double)((2 * k - 1) * (2 * k));
        sum += term;
    }
    return sum;
}

constexpr double sin_oct(double a);
constexpr double cos_oct(double a) {        // a in [0, 2 pi]
    return a > kPiC           ? cos_oct(2.0 * kPiC - a)
           : a > kPiC / 2     ? -cos_oct(kPiC - a)
           : a > kPiC / 4     ? sin_oct(kPiC / 2 - a)
                              : taylor_cos(a);
}
constexpr double sin_oct(double a) {
    return a > kPiC           ? -sin_oct(2.0 * kPiC - a)
           : a > kPiC / 2     ? sin_oct(kPiC - a)
           : a > kPiC / 4     ? cos_oct(kPiC / 2 - a)
                              : taylor_sin(a);
}

// exp(-2 pi i m / N) for m = 0..N-1 (the forward DFT's root powers)
template <int N, typename T>
struct RootTab {
    T c[N], s[N];
    constexpr RootTab() : c(), s() {
        for (int m = 0; m < N; ++m) {
            // exact zeros and ones at the quarter turns
            if (4 * m == N || 4 * m == 3 * N) c[m] = (T)0;
            else c[m] = (T)cos_oct(2.0 * kPiC * (double)m / (double)N);
            if (2 * m == N || m == 0) s[m] = (T)0;
            else s[m] = (T)-sin_oct(2.0 * kPiC * (double)m / (double)N);
        }
    }
};

// ---- codelets: in-place DFT of N registers, natural order in and out ------
template <int N>
__host__ __device__ constexpr int codelet_split() {     // first factor P of a composite N = P * Q
    return N % 4 == 0 ? 4 : N % 2 == 0 ? 2 : N % 3 == 0 ? 3 : N % 5 == 0 ? 5 : 7;
}

template <int N>
__host__ __device__ constexpr bool codelet_base() {
    return N == 1 || N == 2 || N == 3 || N == 4 || N == 5 || N == 7 || N == 8;
}

template <int N, bool INV, typename T>
__device__ __forceinline__ void dftr(cx<T> *v);

template <int N, bool INV, typename T>
__device__ __forceinline__ void dftr_composite(cx<T> *v) {
    constexpr int P = codelet_split<N>();
    constexpr int Q = N / P;
    constexpr RootTab<N, T> W{};
    cx<T> w[N];   // w[k1 * Q + q]: length-P transform of column q, twiddled
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        cx<T> u[P];
#pragma unroll
        for (int p = 0; p < P; ++p) u[p] = v[q + Q * p];
        dftr<P, INV>(u);
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
            const int m = q * k1;
            if (m != 0) {
                const T c = W.c[m], s = INV ? -W.s[m] : W.s[m];
                u[k1] = cx<T>{u[k1].x * c - u[k1].y * s, u[k1].x * s + u[k1].y * c};
            }
            w[k1 * Q + q] = u[k1];
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
        cx<T> z[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) z[q] = w[k1 * Q + q];
        dftr<Q, INV>(z);
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) v[k1 + P * k2] = z[k2];
    }
}

template <int N, bool INV, typename T>
__device__ __forceinline__ void dftr(cx<T> *v) {
    if constexpr (N == 1) {
    } else if constexpr (codelet_base<N>()) {
        dft<N, INV>(v);
    } else {
        dftr_composite<N, INV>(v);
    }
}

// ---- two-pass transform of `nlines` lines in shared memory ---------------
// a: data (element i of line l at a[i * ld + l]), overwritten by the result;
// b: scratch of the same shape; tw: exp(-2 pi i m / N), m < N (forward).
// All threads of the block must call; ends with a barrier.
template <int N1, int N2, bool INV, typename T>
__device__ __noinline__ void fft2p(cx<T> *a, cx<T> *b, int nlines, int ld, const cx<T> *tw) {
    constexpr int N = N1 * N2;
    const int nt = blockDim.x;
    const int dl = nt % nlines, dj = nt / nlines;
    {
        int l = threadIdx.x % nlines, j2 = threadIdx.x / nlines;
        for (; j2 < N2;) {
            cx<T> v[N1];
            const cx<T> *src = a + (size_t)j2 * ld + l;
#pragma unroll
            for (int j1 = 0; j1 < N1; ++j1) v[j1] = src[(size_t)j1 * N2 * ld];
            dftr<N1, INV>(v);
#pragma unroll
            for (int k1 = 1; k1 < N1; ++k1) {
                cx<T> w = tw[j2 * k1];
                if (INV) w.y = -w.y;
                v[k1] = cmul(v[k1], w);
            }
            cx<T> *dst = b + (size_t)j2 * ld + l;
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) dst[(size_t)k1 * N2 * ld] = v[k1];
            l += dl;
            j2 += dj;
            if (l >= nlines) {
                l -= nlines;
                ++j2;
            }
        }
    }
    __syncthreads();
    {
        int l = threadIdx.x % nlines, k1 = threadIdx.x / nlines;
        for (; k1 < N1;) {
            cx<T> v[N2];
            const cx<T> *src = b + (size_t)k1 * N2 * ld + l;
#pragma unroll
            for (int j2 = 0; j2 < N2; ++j2) v[j2] = src[(size_t)j2 * ld];
            dftr<N2, INV>(v);
            cx<T> *dst = a + (size_t)k1 * ld + l;
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) dst[(size_t)k2 * N1 * ld] = v[k2];
            l += dl;
            k1 += dj;
            if (l >= nlines) {
                l -= nlines;
                ++k1;
            }
        }
    }
    __syncthreads();
    (void)N;
}

// Transform `nlines` lines of length p.n (layout [i][ld]); returns the buffer
// holding the result (a or b).  FP32 lengths with a compiled two-pass split
// use fft2p, all others the generic Stockham stages.  Ends with a barrier.
template <bool INV, typename T>
__device__ __forceinline__ cx<T> *fft_auto(cx<T> *a, cx<T> *b, const AxisPlan &p, int nlines, int ld,
                                           const cx<T> *tw) {
    if constexpr (sizeof(T) == 4) {
        switch (p.n) {
            case 16: fft2p<4, 4, INV>(a, b, nlines, ld, tw); return a;
            case 24: fft2p<8, 3, INV>(a, b, nlines, ld, tw); return a;
            case 32: fft2p<8, 4, INV>(a, b, nlines, ld, tw); return a;
            case 40: fft2p<8, 5, INV>(a, b, nlines, ld, tw); return a;
            case 48: fft2p<8, 6, INV>(a, b, nlines, ld, tw); return a;
            case 64: fft2p<8, 8, INV>(a, b, nlines, ld, tw); return a;
            case 72: fft2p<8, 9, INV>(a, b, nlines, ld, tw); return a;
            case 80: fft2p<10, 8, INV>(a, b, nlines, ld, tw); return a;
            case 96: fft2p<12, 8, INV>(a, b, nlines, ld, tw); return a;
            case 112: fft2p<14, 8, INV>(a, b, nlines, ld, tw); return a;
            case 128: fft2p<16, 8, INV>(a, b, nlines, ld, tw); return a;
            case 144: fft2p<12, 12, INV>(a, b, nlines, ld, tw); return a;
            case 160: fft2p<16, 10, INV>(a, b, nlines, ld, tw); return a;
            case 192: fft2p<16, 12, INV>(a, b, nlines, ld, tw); return a;
            case 224: fft2p<16, 14, INV>(a, b, nlines, ld, tw); return a;
            case 256: fft2p<16, 16, INV>(a, b, nlines, ld, tw); return a;
            default: break;
        }
    }
    return fft_lines<INV>(a, b, p, nlines, ld, tw);
}

// ---- in-place transforms with a permuted spectrum --------------------------
// Forward: natural input; position p = k1 N2 + k2 of the result holds
// frequency k1 + N1 k2.  Inverse: takes that permuted order, returns natural
// order.  Both passes of either direction read and write the same positions
// per work item, so no scratch buffer is needed.  Layout [i][ld] as above.
__host__ __device__ constexpr int fft_split(int n) {   // N1 of the two-pass split, 0: none
    return n == 16 ? 4 : n == 24 ? 8 : n == 32 ? 8 : n == 40 ? 8 : n == 48 ? 8 : n == 64 ? 8 : n == 72 ? 8
         : n == 80 ? 10 : n == 96 ? 12 : n == 112 ? 14 : n == 128 ? 16 : n == 144 ? 12 : n == 160 ? 16
         : n == 192 ? 16 : n == 224 ? 16 : n == 256 ? 16 : 0;
}

// frequency held at position p of a permuted spectrum of length n1 * n2
__host__ __device__ inline int fft_perm_freq(int p, int n1, int n2) { return p / n2 + n1 * (p % n2); }

// position of frequency f in a permuted spectrum of length n1 * n2
__host__ __device__ inline int fft_perm_pos(int f, int n1, int n2) { return (f % n1) * n2 + f / n1; }

// frequency index at position p of an axis of length n whose forward pass
// left the permuted order (n1 = its split), or p itself (n1 = 0)
__host__ __device__ inline int axis_freq(int p, int n, int n1) { return n1 ? fft_perm_freq(p, n1, n / n1) : p; }

template <int N1, int N2, bool INV, typename T>
__device__ __noinline__ void fft_ip(cx<T> *a, int nlines, int ld, const cx<T> *tw) {
    const int nt = blockDim.x;
    const int dl = nt % nlines, dj = nt / nlines;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        // forward: strided pass then block pass; inverse: block pass then strided pass
        const bool strided = (pass == 0) != INV;
        int l = threadIdx.x % nlines, q = threadIdx.x / nlines;
        if (strided) {
            for (; q < N2;) {                 // item (l, j2): positions j1 N2 + j2
                cx<T> v[N1];
                cx<T> *p = a + (size_t)q * ld + l;
#pragma unroll
                for (int j1 = 0; j1 < N1; ++j1) v[j1] = p[(size_t)j1 * N2 * ld];
                dftr<N1, INV>(v);
                if (!INV) {
#pragma unroll
                    for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], tw[q * k1]);
                }
#pragma unroll
                for (int j1 = 0; j1 < N1; ++j1) p[(size_t)j1 * N2 * ld] = v[j1];
                l += dl;
                q += dj;
                if (l >= nlines) {
                    l -= nlines;
                    ++q;
                }
            }
        } else {
            for (; q < N1;) {                 // item (l, k1): positions k1 N2 + j2
                cx<T> v[N2];
                cx<T> *p = a + (size_t)q * N2 * ld + l;
#pragma unroll
                for (int j2 = 0; j2 < N2; ++j2) v[j2] = p[(size_t)j2 * ld];
                dftr<N2, INV>(v);
                if (INV) {
#pragma unroll
                    for (int j2 = 1; j2 < N2; ++j2) {
                        cx<T> w = tw[q * j2];
                        w.y = -w.y;
                        v[j2] = cmul(v[j2], w);
                    }
                }
#pragma unroll
                for (int j2 = 0; j2 < N2; ++j2) p[(size_t)j2 * ld] = v[j2];
                l += dl;
                q += dj;
                if (l >= nlines) {
                    l -= nlines;
                    ++q;
                }
            }
        }
        __syncthreads();
    }
}

// In-place permuted transform of `nlines` lines of length n (an fft_split
// length); all threads of the block call; ends with a barrier.
template <bool INV, typename T>
__device__ __forceinline__ void fft_ip_auto(cx<T> *a, int n, int nlines, int ld, const cx<T> *tw) {
    switch (n) {
        case 16: fft_ip<4, 4, INV>(a, nlines, ld, tw); break;
        case 24: fft_ip<8, 3, INV>(a, nlines, ld, tw); break;
        case 32: fft_ip<8, 4, INV>(a, nlines, ld, tw); break;
        case 40: fft_ip<8, 5, INV>(a, nlines, ld, tw); break;
        case 48: fft_ip<8, 6, INV>(a, nlines, ld, tw); break;
        case 64: fft_ip<8, 8, INV>(a, nlines, ld, tw); break;
        case 72: fft_ip<8, 9, INV>(a, nlines, ld, tw); break;
        case 80: fft_ip<10, 8, INV>(a, nlines, ld, tw); break;
        case 96: fft_ip<12, 8, INV>(a, nlines, ld, tw); break;
        case 112: fft_ip<14, 8, INV>(a, nlines, ld, tw); break;
        case 128: fft_ip<16, 8, INV>(a, nlines, ld, tw); break;
        case 144: fft_ip<12, 12, INV>(a, nlines, ld, tw); break;
        case 160: fft_ip<16, 10, INV>(a, nlines, ld, tw); break;
        case 192: fft_ip<16, 12, INV>(a, nlines, ld, tw); break;
        case 224: fft_ip<16, 14, INV>(a, nlines, ld, tw); break;
        case 256: fft_ip<16, 16, INV>(a, nlines, ld, tw); break;
        default: break;
    }
}

// The x / y passes also split 640-point axes (the paper's density grid), as
// 32 x 20: their blocks hold the registers of a 32-point codelet (two blocks
// per SM), which the z passes, at three blocks per SM, do not.
__host__ __device__ constexpr int xy_split(int n) { return n == 640 ? 32 : fft_split(n); }

// In-place permuted transform of the x / y passes (an xy_split length).
template <bool INV, typename T>
__device__ __forceinline__ void fft_ip_xy_auto(cx<T> *a, int n, int nlines, int ld, const cx<T> *tw) {
    if (n == 640) fft_ip<32, 20, INV>(a, nlines, ld, tw);
    else fft_ip_auto<INV>(a, n, nlines, ld, tw);
}

// Inverse in-place permuted transform of a z tile whose input is the staged
// half spectrum of the 20 real fields, packed into complex lines on the fly:
// line l = 10 li + c holds Z(f) = X_2c(f) + i X_2c+1(f) for f < nzh (the
// imaginary parts of the f = 0 and Nyquist bins dropped) and the Hermitian
// mirror conj(X_2c(nz - f)) + i conj(X_2c+1(nz - f)) above.  spec: [li][kz][20]
// complex (16-byte aligned).  The first (block) pass reads its N2 inputs at
// frequencies q + N1 j2 straight from spec and writes positions q N2 + j2 of
// a; the second pass is that of fft_ip.  Natural order in a at the end;
// ends with a barrier.
template <int N1, int N2, typename T>
__device__ __noinline__ void fft_ip_inv_packed(cx<T> *a, const cx<T> *spec, int nlines, int ld, int nzh,
                                               const cx<T> *tw) {
    constexpr int N = N1 * N2;
    const int nt = blockDim.x;
    const int dl = nt % nlines, dj = nt / nlines;
    {
        int l = threadIdx.x % nlines, q = threadIdx.x / nlines;
        for (; q < N1;) {                     // item (l, q): positions q N2 + j2
            const int li = l / 10, c = l - 10 * li;
            const cx<T> *sl = spec + (size_t)li * nzh * NQ + 2 * c;
            cx<T> v[N2];
#pragma unroll
            for (int j2 = 0; j2 < N2; ++j2) {
                const int f = q + N1 * j2;
                const bool mirror = f >= nzh;
                const int kz = mirror ? N - f : f;
                cx<T> x0 = sl[(size_t)kz * NQ], x1 = sl[(size_t)kz * NQ + 1];
                if (f == 0 || ((N & 1) == 0 && f == N / 2)) {
                    x0.y = (T)0;
                    x1.y = (T)0;
                }
                v[j2] = mirror ? cx<T>{x0.x + x1.y, x1.x - x0.y} : cx<T>{x0.x - x1.y, x0.y + x1.x};
            }
            dftr<N2, true>(v);
#pragma unroll
            for (int j2 = 1; j2 < N2; ++j2) {
                cx<T> w = tw[q * j2];
                w.y = -w.y;
                v[j2] = cmul(v[j2], w);
            }
            cx<T> *p = a + (size_t)q * N2 * ld + l;
#pragma unroll
            for (int j2 = 0; j2 < N2; ++j2) p[(size_t)j2 * ld] = v[j2];
            l += dl;
            q += dj;
            if (l >= nlines) {
                l -= nlines;
                ++q;
            }
        }
    }
    __syncthreads();
    {
        int l = threadIdx.x % nlines, q = threadIdx.x / nlines;
        for (; q < N2;) {                     // item (l, j2): positions j1 N2 + j2
            cx<T> v[N1];
            cx<T> *p = a + (size_t)q * ld + l;
#pragma unroll
            for (int j1 = 0; j1 < N1; ++j1) v[j1] = p[(size_t)j1 * N2 * ld];
            dftr<N1, true>(v);
#pragma unroll
            for (int j1 = 0; j1 < N1; ++j1) p[(size_t)j1 * N2 * ld] = v[j1];
            l += dl;
            q += dj;
            if (l >= nlines) {
                l -= nlines;
                ++q;
            }
        }
    }
    __syncthreads();
}

// Forward in-place transform of a z tile of complex lines l = 10 li + c
// (Z = theta_2c + i theta_2c+1, natural order in a) whose second pass writes
// the two real spectra straight to the half spectrum out ([li][kz][20]
// complex, global): item (l, k1) transforms the blocks k1 and N1 - k1 together,
// whose frequencies k1 + N1 k2 and N1 - k1 + N1 k2' are each other's mirrors
// nz - f, and writes X_2c(f) = (Z(f) + conj Z(-f)) / 2 and
// X_2c+1(f) = (Z(f) - conj Z(-f)) / 2i for every f < nzh of the two blocks.
// a is left in an intermediate state; ends without a barrier (the caller
// synchronises before a is reused).
template <typename T>
__device__ __forceinline__ void unpack_store(cx<T> *out, cx<T> z, cx<T> zm) {
    const T ex = (T)0.5 * (z.x + zm.x), ey = (T)0.5 * (z.y - zm.y);
    const T ox = (T)0.5 * (z.y + zm.y), oy = (T)-0.5 * (z.x - zm.x);
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(out) = make_float4(ex, ey, ox, oy);
    } else {
        out[0] = cx<T>{ex, ey};
        out[1] = cx<T>{ox, oy};
    }
}

template <int N1, int N2, typename T>
__device__ __noinline__ void fft_ip_fwd_unpack(cx<T> *a, cx<T> *out, int nlines, int ld, int nzh, const cx<T> *tw) {
    const int nt = blockDim.x;
    const int dl = nt % nlines, dj = nt / nlines;
    {
        // first pass as fft_ip (forward: strided, then twiddles)
        int l = threadIdx.x % nlines, q = threadIdx.x / nlines;
        for (; q < N2;) {
            cx<T> v[N1];
            cx<T> *p = a + (size_t)q * ld + l;
#pragma unroll
            for (int j1 = 0; j1 < N1; ++j1) v[j1] = p[(size_t)j1 * N2 * ld];
            dftr<N1, false>(v);
#pragma unroll
            for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], tw[q * k1]);
#pragma unroll
            for (int j1 = 0; j1 < N1; ++j1) p[(size_t)j1 * N2 * ld] = v[j1];
            l += dl;
            q += dj;
            if (l >= nlines) {
                l -= nlines;
                ++q;
            }
        }
    }
    __syncthreads();
    constexpr int NH = N1 / 2 + 1;   // block pairs (k1, N1 - k1), k1 = 0 .. N1/2
    int l = threadIdx.x % nlines, q = threadIdx.x / nlines;
    for (; q < NH;) {
        const int k1 = q, k1p = (N1 - k1) % N1;
        const int li = l / 10, c = l - 10 * li;
        cx<T> *ol = out + (size_t)li * nzh * NQ + 2 * c;
        cx<T> u[N2], w[N2];
        {
            const cx<T> *p = a + (size_t)k1 * N2 * ld + l;
#pragma unroll
            for (int j2 = 0; j2 < N2; ++j2) u[j2] = p[(size_t)j2 * ld];
            dftr<N2, false>(u);                  // u[k2] = Z(k1 + N1 k2)
        }
        if (k1 == 0) {
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                const int f = N1 * k2;
                if (f < nzh) unpack_store(ol + (size_t)f * NQ, u[k2], u[(N2 - k2) % N2]);
            }
        } else if (k1p == k1) {                  // k1 = N1 / 2
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                const int f = k1 + N1 * k2;
                if (f < nzh) unpack_store(ol + (size_t)f * NQ, u[k2], u[N2 - 1 - k2]);
            }
        } else {
            {
                const cx<T> *p = a + (size_t)k1p * N2 * ld + l;
#pragma unroll
                for (int j2 = 0; j2 < N2; ++j2) w[j2] = p[(size_t)j2 * ld];
                dftr<N2, false>(w);              // w[k2] = Z(N1 - k1 + N1 k2)
            }
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                const int f = k1 + N1 * k2, fp = k1p + N1 * k2;
                if (f < nzh) unpack_store(ol + (size_t)f * NQ, u[k2], w[N2 - 1 - k2]);
                if (fp < nzh) unpack_store(ol + (size_t)fp * NQ, w[k2], u[N2 - 1 - k2]);
            }
        }
        l += dl;
        q += dj;
        if (l >= nlines) {
            l -= nlines;
            ++q;
        }
    }
}

template <typename T>
__device__ __forceinline__ void fft_ip_fwd_unpack_auto(cx<T> *a, cx<T> *out, int n, int nlines, int ld, int nzh,
                                                       const cx<T> *tw) {
    switch (n) {
        case 16: fft_ip_fwd_unpack<4, 4>(a, out, nlines, ld, nzh, tw); break;
        case 24: fft_ip_fwd_unpack<8, 3>(a, out, nlines, ld, nzh, tw); break;
        case 32: fft_ip_fwd_unpack<8, 4>(a, out, nlines, ld, nzh, tw); break;
        case 40: fft_ip_fwd_unpack<8, 5>(a, out, nlines, ld, nzh, tw); break;
        case 48: fft_ip_fwd_unpack<8, 6>(a, out, nlines, ld, nzh, tw); break;
        case 64: fft_ip_fwd_unpack<8, 8>(a, out, nlines, ld, nzh, tw); break;
        case 72: fft_ip_fwd_unpack<8, 9>(a, out, nlines, ld, nzh, tw); break;
        case 80: fft_ip_fwd_unpack<10, 8>(a, out, nlines, ld, nzh, tw); break;
        case 96: fft_ip_fwd_unpack<12, 8>(a, out, nlines, ld, nzh, tw); break;
        case 112: fft_ip_fwd_unpack<14, 8>(a, out, nlines, ld, nzh, tw); break;
        case 128: fft_ip_fwd_unpack<16, 8>(a, out, nlines, ld, nzh, tw); break;
        case 144: fft_ip_fwd_unpack<12, 12>(a, out, nlines, ld, nzh, tw); break;
        case 160: fft_ip_fwd_unpack<16, 10>(a, out, nlines, ld, nzh, tw); break;
        case 192: fft_ip_fwd_unpack<16, 12>(a, out, nlines, ld, nzh, tw); break;
        case 224: fft_ip_fwd_unpack<16, 14>(a, out, nlines, ld, nzh, tw); break;
        case 256: fft_ip_fwd_unpack<16, 16>(a, out, nlines, ld, nzh, tw); break;
        default: break;
    }
}

template <typename T>
__device__ __forceinline__ void fft_ip_inv_packed_auto(cx<T> *a, const cx<T> *spec, int n, int nlines, int ld,
                                                       int nzh, const cx<T> *tw) {
    switch (n) {
        case 16: fft_ip_inv_packed<4, 4>(a, spec, nlines, ld, nzh, tw); break;
        case 24: fft_ip_inv_packed<8, 3>(a, spec, nlines, ld, nzh, tw); break;
        case 32: fft_ip_inv_packed<8, 4>(a, spec, nlines, ld, nzh, tw); break;
        case 40: fft_ip_inv_packed<8, 5>(a, spec, nlines, ld, nzh, tw); break;
        case 48: fft_ip_inv_packed<8, 6>(a, spec, nlines, ld, nzh, tw); break;
        case 64: fft_ip_inv_packed<8, 8>(a, spec, nlines, ld, nzh, tw); break;
        case 72: fft_ip_inv_packed<8, 9>(a, spec, nlines, ld, nzh, tw); break;
        case 80: fft_ip_inv_packed<10, 8>(a, spec, nlines, ld, nzh, tw); break;
        case 96: fft_ip_inv_packed<12, 8>(a, spec, nlines, ld, nzh, tw); break;
        case 112: fft_ip_inv_packed<14, 8>(a, spec, nlines, ld, nzh, tw); break;
        case 128: fft_ip_inv_packed<16, 8>(a, spec, nlines, ld, nzh, tw); break;
        case 144: fft_ip_inv_packed<12, 12>(a, spec, nlines, ld, nzh, tw); break;
        case 160: fft_ip_inv_packed<16, 10>(a, spec, nlines, ld, nzh, tw); break;
        case 192: fft_ip_inv_packed<16, 12>(a, spec, nlines, ld, nzh, tw); break;
        case 224: fft_ip_inv_packed<16, 14>(a, spec, nlines, ld, nzh, tw); break;
        case 256: fft_ip_inv_packed<16, 16>(a, spec, nlines, ld, nzh, tw); break;
        default: break;
    }
}

}  // namespace vdwgb
