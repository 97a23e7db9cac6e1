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
#include "tma.cuh"
#include "dfloat.cuh"
#include "dfmath.cuh"
#include "fftreg.cuh"
#include "contract.cuh"

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

// ---------------------------------------------------------------------------
// q0 for the FP32-mixed form in double-float arithmetic (about 46 bits;
// GB300's FP64 pipe runs at 1/64 of its FP32 rate).  Same formulas as
// q0_point, organised for few operations; the elementary functions and the
// saturation are those of dfmath.cuh.
// ---------------------------------------------------------------------------
struct Q0M {
    bool live;
    int j;
    float B;
    float dqdn, dqds;
    float nf;        // n rounded to FP32
    double q0;
};

struct Q0Tab {
    dfl qd[NQ];          // the q mesh and 1/h in double-float
    dfl invhd[NQ];
    float4 lnt[64];      // {1/c_i in FP32, ln c_i hi, ln c_i lo, 0}
    float2 ex2[64];      // 2^(-j/64) hi, lo
};

__device__ __forceinline__ void load_q0tab(Q0Tab *t) {
    load_df_tables(t->lnt, t->ex2);
    for (int i = threadIdx.x; i < NQ; i += blockDim.x) {
        t->qd[i] = df_from(c_qm.q[i]);
        t->invhd[i] = df_from(c_qm.invh[i]);
    }
}

// interval j with q_j <= q0 < q_{j+1} and B = (q0 - q_j) / h_j of a
// double-float q0; q0 below q_min: j = 0, B = 0, q0 = q_min and false (the
// derivatives stay zero)
__device__ __forceinline__ bool df_interval(dfl q0, const Q0Tab *tb, Q0M &r) {
    const dfl qmin = tb->qd[0];
    if (df_lt(q0, qmin)) {
        r.j = 0;
        r.B = 0.f;
        r.q0 = c_qm.q_min;
        return false;
    }
    r.q0 = df_to(q0);
    int lo = 0, hi = NQ - 2;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (df_lt(q0, tb->qd[mid])) hi = mid - 1;
        else lo = mid;
    }
    r.j = lo;
    const dfl qj = tb->qd[lo];
    r.B = ((q0.hi - qj.hi) + (q0.lo - qj.lo)) * tb->invhd[lo].hi;
    return true;
}

// zc = -Z_ab / 36 in double-float (positive)
__device__ __forceinline__ Q0M q0_point_df(double n, double s, dfl zc, const Q0Tab *tb) {
    Q0M r;
    // n > n_min and sigma < 0 -> 0 compared as integers (IEEE order of
    // non-negative doubles), keeping the FP64 pipe free
    r.live = __double_as_longlong(n) > __double_as_longlong(c_qm.n_min);
    r.dqdn = 0.f;
    r.dqds = 0.f;
    r.nf = 0.f;
    if (!r.live) {
        r.j = -1;
        r.B = 0.f;
        r.q0 = c_qm.q_min;
        return r;
    }
    if (__double_as_longlong(s) <= 0) s = 0.0;
    const double A = 0.031091, a1 = 0.2137;
    const double b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
    const double PI = 3.14159265358979323846;
    const dfl nd = df_from_bits(n), sd = df_from_bits(s);
    r.nf = nd.hi + nd.lo;
    const dfl kF = df_cbrt(df_mul(nd, DF(3.0 * PI * PI)));
    const dfl ikF = df_rcp_fast(kF);
    const dfl rs = df_mul(ikF, DF(1.9191582926775128));      // (9 pi / 4)^(1/3) / k_F
    const dfl srs = df_sqrt(rs);
    dfl poly = df_add_pos(df_mul(DF(b4), srs), DF(b3));
    poly = df_add_pos(df_mul(poly, srs), DF(b2));
    poly = df_add_pos(df_mul(poly, srs), DF(b1));
    const dfl D = df_mul(df_mul(poly, srs), DF(2.0 * A));   // 2A (b1 rs^1/2 + b2 rs + b3 rs^3/2 + b4 rs^2)
    const dfl L = df_log1p(df_rcp_fast(D), tb->lnt);
    const dfl ar = df_add_pos(DF(1.0), df_mul(DF(a1), rs));
    const dfl meps = df_mul(df_mul(DF(2.0 * A), ar), L);    // -eps_c > 0
    const dfl in2 = df_rcp_fast(df_mul(nd, nd));
    const dfl G = df_mul(df_mul(df_mul(zc, sd), ikF), in2);  // gradient term >= 0
    const dfl qraw = df_add_pos(df_add_pos(kF, df_mul(DF(4.0 * PI / 3.0), meps)), G);
    const dfl t = df_mul(qraw, DF(0.2));
    float dh = 0.f;
    const dfl q0 = df_saturate(t, 5.0f, tb->ex2, dh);
    if (!df_interval(q0, tb, r)) return r;
    if (dh == 0.f) return r;
    // dq_raw/dn = (k_F/3 + (4 pi/9) r_s deps/dr_s - (7/3) G) / n; the sum can
    // cancel, so it is formed in double-float; dq_raw/dsigma is a plain product
    const dfl isrs = df_mul(srs, df_mul(kF, DF(1.0 / 1.9191582926775128)));   // r_s^(-1/2)
    dfl dD = df_add_pos(df_mul(DF(0.5 * b1), isrs), DF(b2));
    dD = df_add_pos(dD, df_mul(DF(1.5 * b3), srs));
    dD = df_add_pos(dD, df_mul(DF(2.0 * b4), rs));
    dD = df_mul(dD, DF(2.0 * A));
    const dfl qd = df_mul(dD, df_rcp_fast(df_mul(D, df_add_pos(D, DF(1.0)))));
    const dfl deps = df_sub(df_mul(df_mul(DF(2.0 * A), ar), qd), df_mul(DF(2.0 * A * a1), L));
    const dfl t12 = df_add(df_mul(kF, DF(1.0 / 3.0)), df_mul(df_mul(DF(4.0 * PI / 9.0), rs), deps));
    const dfl dqn = df_mul(df_sub(t12, df_mul(DF(7.0 / 3.0), G)), df_rcp_fast(nd));
    r.dqdn = dh * dqn.hi;
    r.dqds = dh * (zc.hi * ikF.hi * in2.hi);
    return r;
}

// q0 formed beforehand (the spin-polarised form): the interval of the given
// q0 at live points, and the records' derivative factors set so that the
// z-inverse pass leaves sum_a F_a p_a in dedn (dq0/dn = 0) and
// n sum_a F_a p'_a in dedsigma (dq0/dsigma = 1)
__device__ __forceinline__ Q0M q0_given_df(double n, double q0, const Q0Tab *tb) {
    Q0M r;
    r.live = __double_as_longlong(n) > __double_as_longlong(c_qm.n_min);
    r.dqdn = 0.f;
    r.dqds = 0.f;
    r.nf = 0.f;
    if (!r.live) {
        r.j = -1;
        r.B = 0.f;
        r.q0 = c_qm.q_min;
        return r;
    }
    const dfl nd = df_from_bits(n);
    r.nf = nd.hi + nd.lo;
    df_interval(df_from_bits(q0), tb, r);
    r.dqds = 1.f;
    return r;
}

__device__ __forceinline__ Q0 q0_given(double n, double q0) {
    Q0 r;
    r.live = n > c_qm.n_min;
    r.q0 = r.live ? q0 : c_qm.q_min;
    r.dqdn = 0.0;
    r.dqds = r.live ? 1.0 : 0.0;
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

// Shared q-mesh tables in precision T.
template <typename T>
struct QShared {
    double q[NQ];
    double invh[NQ];
    Q0Tab q0t;       // double-float mesh and ln / exp tables (FP32-mixed q0)
    T h[NQ];
    T hh6[NQ];       // h_j^2 / 6
    T h6[NQ];        // h_j / 6
    T ih[NQ];        // 1 / h_j
    alignas(16) T d2[NQ * NQ];
};

template <typename T>
__device__ __forceinline__ void load_qshared(QShared<T> *qs) {
    for (int i = threadIdx.x; i < NQ * NQ; i += blockDim.x) qs->d2[i] = (T)c_qm.d2[i];
    load_q0tab(&qs->q0t);
    for (int i = threadIdx.x; i < NQ; i += blockDim.x) {
        qs->q[i] = c_qm.q[i];
        qs->invh[i] = c_qm.invh[i];
        qs->h[i] = (T)c_qm.h[i];
        qs->hh6[i] = (T)(c_qm.h[i] * c_qm.h[i] / 6.0);
        qs->h6[i] = (T)(c_qm.h[i] / 6.0);
        qs->ih[i] = (T)c_qm.invh[i];
    }
}

__device__ __forceinline__ size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// z-forward: theta and the real-to-complex transform along z.
// Two real fields share one complex line: c = theta_{2m} + i theta_{2m+1}.
// A tile is LZ consecutive (x, y) lines; in shared memory element z of
// complex line li * 10 + c sits at buf[z * ld + li * 10 + c], with an odd
// row stride ld so that threads on consecutive z hit different banks.
// ---------------------------------------------------------------------------

// Rows j and j + 1 of the helper-spline second-derivative table.
template <typename T>
__device__ __forceinline__ void d2_rows(int j, const T *d2s, T *r0, T *r1) {
    if constexpr (sizeof(T) == 4) {
        const float4 *a = reinterpret_cast<const float4 *>(d2s + j * NQ);
#pragma unroll
        for (int k = 0; k < NQ / 4; ++k) {
            const float4 u = a[k], v = a[k + NQ / 4];
            r0[4 * k] = u.x; r0[4 * k + 1] = u.y; r0[4 * k + 2] = u.z; r0[4 * k + 3] = u.w;
            r1[4 * k] = v.x; r1[4 * k + 1] = v.y; r1[4 * k + 2] = v.z; r1[4 * k + 3] = v.w;
        }
    } else {
        const double2 *a = reinterpret_cast<const double2 *>(d2s + j * NQ);
#pragma unroll
        for (int k = 0; k < NQ / 2; ++k) {
            const double2 u = a[k], v = a[k + NQ / 2];
            r0[2 * k] = u.x; r0[2 * k + 1] = u.y;
            r1[2 * k] = v.x; r1[2 * k + 1] = v.y;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) k_zfwd(const SysDev *__restrict__ sys, const int *__restrict__ prefix,
                                              int nsys, int total) {
    extern __shared__ __align__(16) unsigned char smem[];
    QShared<T> *qs = reinterpret_cast<QShared<T> *>(smem);
    unsigned char *base = smem + align_up(sizeof(QShared<T>), 16);
    load_qshared(qs);
    const int nt = blockDim.x;
    __shared__ SysDev sS;                    // descriptor of the current tile's system
    int cur_sys = -1, tbase = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int nsi = advance_sys(prefix, nsys, t, cur_sys);
        const bool changed = nsi != cur_sys;
        if (changed) {
            __syncthreads();                 // readers of the previous descriptor are done
            copy_sys(&sS, &sys[nsi]);
            __syncthreads();
            cur_sys = nsi;
            tbase = prefix[nsi];
        }
        const SysDev &S = sS;
        const int lt = t - tbase;
        const int nz = S.nz, nzh = S.nzh, LZ = S.LZ;
        const int nlines_tot = S.nx * S.ny;
        const int l0 = lt * LZ;
        const int nl = min(LZ, nlines_tot - l0);
        if (!VDWGB_OK(lt >= 0 && l0 >= 0 && nl >= 1, S.err)) continue;   // tile past the system's lines
        const int L = 10 * nl;              // complex lines in this tile
        const int ld = z_ld(nl);
        cx<T> *tw = reinterpret_cast<cx<T> *>(base);
        cx<T> *bufA = tw + ((nz + 1) & ~1);
        cx<T> *bufB = bufA + (size_t)nz * ld;
        if (changed) {
            const cx<T> *twg = reinterpret_cast<const cx<T> *>(S.tw[2]);
            for (int i = threadIdx.x; i < nz; i += nt) tw[i] = twg[i];
            __syncthreads();   // q tables and twiddles ready
        }
        Rec<T> *rec = reinterpret_cast<Rec<T> *>(S.rec);
        const size_t p0 = (size_t)l0 * nz;
        const double *gn = S.n + p0, *gs = S.sigma + p0;
        const dfl zc = dfl{S.zc[0], S.zc[1]};
        {
            // points i = li * nz + z, walked without division
            const int dz = nt % nz, dli = nt / nz;
            int z = threadIdx.x % nz, li = threadIdx.x / nz;
            {
                // the next tile's n and sigma lines into L2 while this tile runs
                const int tn = t + gridDim.x;
                if (tn < total && tn < tbase + S.tiles[0]) {
                    const int l0n = (tn - tbase) * LZ;
                    const int nln = min(LZ, nlines_tot - l0n);
                    const size_t bytes = (size_t)nln * nz * sizeof(double);
                    const char *pn = reinterpret_cast<const char *>(S.n + (size_t)l0n * nz);
                    const char *ps = reinterpret_cast<const char *>(S.sigma + (size_t)l0n * nz);
                    for (size_t o = (size_t)threadIdx.x * 128; o < bytes; o += (size_t)nt * 128) {
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(pn + o));
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(ps + o));
                    }
                }
            }
            // n and sigma are loaded one point ahead, so that the global-memory
            // latency of the next point overlaps q0 of this one
            double n_next = 0.0, s_next = 0.0;
            if (li < nl) {
                n_next = gn[li * nz + z];
                s_next = gs[li * nz + z];
            }
            for (; li < nl;) {
                const int i = li * nz + z;
                const double n = n_next;
                const double sg = s_next;
                {
                    int z2 = z + dz, li2 = li + dli;   // the walk's next point
                    if (z2 >= nz) {
                        z2 -= nz;
                        ++li2;
                    }
                    if (li2 < nl) {
                        n_next = gn[li2 * nz + z2];
                        s_next = gs[li2 * nz + z2];
                    }
                }
                Rec<T> r;
                int j = -1;
                T B = (T)0, ndqn = (T)0, ndqs = (T)0, nn = (T)0;
                if (sizeof(T) == 4) {
                    const Q0M q = S.q0in ? q0_given_df(n, sg, &qs->q0t) : q0_point_df(n, sg, zc, &qs->q0t);
                    j = q.j;
                    B = (T)q.B;
                    nn = (T)q.nf;
                    ndqn = (T)(q.nf * q.dqdn);
                    ndqs = (T)(q.nf * q.dqds);
                } else {
                    nn = (T)n;
                    const Q0 q = S.q0in ? q0_given(n, sg) : q0_point(n, sg, S.Z);
                    if (q.live) {
                        j = q_interval(q.q0, qs->q);
                        B = (T)((q.q0 - qs->q[j]) * qs->invh[j]);
                        ndqn = (T)(n * q.dqdn);
                        ndqs = (T)(n * q.dqds);
                    }
                }
                cx<T> *dst = bufA + (size_t)z * ld + li * 10;
                if (j >= 0) {
                    // theta_a = n p_a: spline part for all a, then the node
                    // terms A [a == j] + B [a == j + 1] at the two dynamic slots
                    T r0[NQ], r1[NQ];
                    d2_rows<T>(j, qs->d2, r0, r1);
                    const T hh6 = qs->hh6[j], A = (T)1 - B;
                    const T cA = nn * (A * A * A - A) * hh6;
                    const T cB = nn * (B * B * B - B) * hh6;
#pragma unroll
                    for (int c = 0; c < 10; ++c)
                        dst[c] = cx<T>{cA * r0[2 * c] + cB * r1[2 * c], cA * r0[2 * c + 1] + cB * r1[2 * c + 1]};
                    T *dt = reinterpret_cast<T *>(dst);
                    const T *d0 = qs->d2 + j * NQ;
                    dt[j] = nn * A + cA * d0[j] + cB * d0[NQ + j];
                    dt[j + 1] = nn * B + cA * d0[j + 1] + cB * d0[NQ + j + 1];
                } else {
#pragma unroll
                    for (int c = 0; c < 10; ++c) dst[c] = cx<T>{(T)0, (T)0};
                }
                r.B = B;
                r.j = j;
                r.ndqn = ndqn;
                r.ndqs = ndqs;
                rec[p0 + i] = r;
                z += dz;
                li += dli;
                if (z >= nz) {
                    z -= nz;
                    ++li;
                }
            }
        }
        __syncthreads();
        // the two real transforms of each line: X_{2c}(kz) = (Z(kz) + conj Z(-kz)) / 2,
        // X_{2c+1}(kz) = (Z(kz) - conj Z(-kz)) / 2i.  FP32 with a split: in
        // place, the second pass writing them straight to the spectrum; other
        // axes: transform, then one thread writes the 10 outputs of half h
        // (c = 5h .. 5h+4) of one (line, kz)
        const int zs = sizeof(T) == 4 ? S.sz1 : 0;
        cx<T> *spec = reinterpret_cast<cx<T> *>(S.spec) + (size_t)l0 * nzh * NQ;
        cx<T> *R = bufA;
        if (zs) fft_ip_fwd_unpack_auto<T>(bufA, spec, nz, L, ld, nzh, tw);
        else R = fft_auto<false>(bufA, bufB, S.ax[2], L, ld, tw);
        if (!zs) {
            const int half = threadIdx.x & 1;
            const int step = nt >> 1;
            const int dk = step % nzh, dli = step / nzh;
            int kz = (threadIdx.x >> 1) % nzh, li = (threadIdx.x >> 1) / nzh;
            for (; li < nl;) {
                const int km = kz == 0 ? 0 : nz - kz;
                const cx<T> *zk = R + (size_t)kz * ld + li * 10 + 5 * half;
                const cx<T> *zm = R + (size_t)km * ld + li * 10 + 5 * half;
                cx<T> *out = spec + ((size_t)li * nzh + kz) * NQ + 10 * half;
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    const cx<T> a = zk[c], b = zm[c];
                    const T ex = (T)0.5 * (a.x + b.x), ey = (T)0.5 * (a.y - b.y);
                    const T ox = (T)0.5 * (a.y + b.y), oy = (T)-0.5 * (a.x - b.x);
                    if constexpr (sizeof(T) == 4) {
                        *reinterpret_cast<float4 *>(out + 2 * c) = make_float4(ex, ey, ox, oy);
                    } else {
                        out[2 * c] = cx<T>{ex, ey};
                        out[2 * c + 1] = cx<T>{ox, oy};
                    }
                }
                kz += dk;
                li += dli;
                if (kz >= nzh) {
                    kz -= nzh;
                    ++li;
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Transforms along y and x.  A tile is (outer index, kz0 .. kz0 + W - 1):
// for the y pass outer = x and the tile's rows run over y; for the x pass
// outer = ky and the rows run over x.  Each row is W * 20 contiguous complex
// values (the [x][y][kz][a] layout), fetched by bulk copies into a double-
// buffered shared-memory stage while the previous tile is transformed.
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

__device__ __forceinline__ float4 ld_row(const float4 *p) { return *p; }
__device__ __forceinline__ dvec4 ld_row(const dvec4 *p) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0];
    const double2 b = reinterpret_cast<const double2 *>(p)[1];
    return make_dvec4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ int fold(int i, int n) { return i <= (n - 1) / 2 ? i : i - n; }

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

struct XYTile {
    int si, lt, nrows, wt, L, ldr, outer, kz0;   // L = wt 20 lines; rows W 20 apart in shared memory
    size_t g0, rowstride;
};

template <bool XPASS>
__device__ __forceinline__ XYTile xy_tile(const SysDev &S, int si, int lt) {
    XYTile g;
    g.si = si;
    g.lt = lt;
    const int W = XPASS ? S.Wx : S.Wy;
    const int ncol = (S.nzh + W - 1) / W;
    g.outer = g.lt / ncol;
    g.kz0 = (g.lt - g.outer * ncol) * W;
    g.wt = min(W, S.nzh - g.kz0);
    g.L = g.wt * NQ;
    g.ldr = W * NQ;
    if (XPASS) {
        g.nrows = S.nx;
        g.g0 = ((size_t)g.outer * S.nzh + g.kz0) * NQ;
        g.rowstride = (size_t)S.ny * S.nzh * NQ;
    } else {
        g.nrows = S.ny;
        g.g0 = ((size_t)g.outer * S.ny * S.nzh + g.kz0) * NQ;
        g.rowstride = (size_t)S.nzh * NQ;
    }
    return g;
}

// warp 0 issues the bulk copies of tile t into buf (completion on bar); the
// tile's system descriptor is `cached` (shared memory) when it is system
// `cached_si`, else read from global memory
template <typename T, bool XPASS>
__device__ __forceinline__ void xy_issue(const SysDev *__restrict__ sys, const int *__restrict__ prefix, int nsys,
                                         int t, cx<T> *buf, unsigned long long *bar, const SysDev *cached = nullptr,
                                         int cached_si = -1, int cached_base = 0) {
    const int si = advance_sys(prefix, nsys, t, cached_si);
    const bool hit = cached && si == cached_si;
    const SysDev &S = hit ? *cached : sys[si];
    const XYTile g = xy_tile<XPASS>(S, si, t - (hit ? cached_base : prefix[si]));
    const cx<T> *spec = reinterpret_cast<const cx<T> *>(S.spec);
    const int lane = threadIdx.x & 31;
    if (!VDWGB_OK(g.outer >= 0 && g.outer < (XPASS ? S.ny : S.nx) && g.kz0 >= 0 && g.wt >= 1, S.err)) {
        if (lane == 0) mbar_expect_tx(bar, 0u);   // complete the phase without copies
        return;
    }
    fence_proxy_async();
    if (S.tmap) {
        // the tile in tensor copies of `nb` rows each (box W 20 x nb; one copy
        // up to 256 rows; columns past the last kz are filled with zeros and
        // never stored back)
        if (lane == 0) {
            const void *map = static_cast<const unsigned char *>(S.tmap) + (XPASS ? 128 : 0);
            int nb = XPASS ? S.tbx : S.tby;
            if (nb < 1 || g.nrows % nb) nb = g.nrows;   // never: the plan divides the rows
            fence_tensormap(map);
            mbar_expect_tx(bar, (unsigned)((size_t)g.ldr * g.nrows * sizeof(cx<T>)));
            for (int r0 = 0; r0 < g.nrows; r0 += nb)
                tma_load_3d(buf + (size_t)r0 * g.ldr, map, g.kz0 * NQ, XPASS ? g.outer : r0, XPASS ? r0 : g.outer,
                            bar);
        }
        return;
    }
    const unsigned rowbytes = (unsigned)(g.L * sizeof(cx<T>));
    if (lane == 0) mbar_expect_tx(bar, rowbytes * (unsigned)g.nrows);
    __syncwarp();
    for (int r = lane; r < g.nrows; r += 32)
        bulk_g2s(buf + (size_t)r * g.ldr, spec + g.g0 + r * g.rowstride, rowbytes, bar);
}

// MODE 0: forward y, 1: inverse y, 2: forward x, 3: inverse x.
// Row tiles cycle through a ring of `nin` input buffers (tile i + nin - 1 is
// requested while tile i is transformed; nin = 1: the next tile is requested
// after this one is stored).  Axes with a compiled two-pass split (FP32)
// transform in place, the forward pass leaving frequencies in the permuted
// order p = k1 N2 + k2 <-> k1 + N1 k2 that the contraction and the inverse
// pass read back; other axes use the scratch buffer (haswork).
template <typename T, int MODE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_xy(const SysDev *__restrict__ sys,
                                                                   const int *__restrict__ prefix, int nsys,
                                                                   int total, int twmax, int bufelems, int nin,
                                                                   int haswork, int *__restrict__ err) {
    constexpr bool XPASS = MODE >= 2;
    constexpr bool INV = (MODE & 1) != 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);   // 128-byte aligned
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem);           // [XY_MAXIN]
    cx<T> *tw = reinterpret_cast<cx<T> *>(smem + XY_HEAD);
    const size_t bstride = xy_buf_stride(bufelems, sizeof(cx<T>));
    unsigned char *in0 = smem + xy_off_in(twmax, sizeof(cx<T>));
    cx<T> *work = reinterpret_cast<cx<T> *>(in0 + (size_t)nin * bstride);
    (void)haswork;
    if (threadIdx.x == 0) {
        for (int k = 0; k < nin; ++k) mbar_init(&bar[k], 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned ph = 0u;              // parity bit per ring slot
    unsigned pending = 0u;         // slots with a requested, not yet consumed tile
    // prologue: tiles 0 .. nin - 2 of this block (nin = 1: tile 0)
    const int pre = nin > 1 ? nin - 1 : 1;
    for (int k = 0; k < pre; ++k) {
        const int tk = blockIdx.x + k * gridDim.x;
        if (tk < total) {
            if (threadIdx.x < 32)
                xy_issue<T, XPASS>(sys, prefix, nsys, tk, reinterpret_cast<cx<T> *>(in0 + (size_t)k * bstride), &bar[k]);
            pending |= 1u << k;
        }
    }
    __shared__ SysDev sS;                    // descriptor of the current tile's system
    int cur_sys = -1, tbase = 0, cur = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int nsi = advance_sys(prefix, nsys, t, cur_sys);
        if (nsi != cur_sys) {
            __syncthreads();                 // readers of the previous descriptor are done
            copy_sys(&sS, &sys[nsi]);
            __syncthreads();
            const cx<T> *twg = reinterpret_cast<const cx<T> *>(sS.tw[XPASS ? 0 : 1]);
            for (int k = threadIdx.x; k < sS.ax[XPASS ? 0 : 1].n; k += blockDim.x) tw[k] = twg[k];
            cur_sys = nsi;
            tbase = prefix[nsi];
        }
        if (nin > 1) {
            // the slot of the previous tile (stored and released at its end)
            const int tn = t + (nin - 1) * gridDim.x;
            const int sn = cur == 0 ? nin - 1 : cur - 1;
            if (tn < total) {
                if (threadIdx.x < 32)
                    xy_issue<T, XPASS>(sys, prefix, nsys, tn, reinterpret_cast<cx<T> *>(in0 + (size_t)sn * bstride),
                                       &bar[sn], &sS, cur_sys, tbase);
                pending |= 1u << sn;
            }
        }
        const SysDev &S = sS;
        const XYTile g = xy_tile<XPASS>(S, nsi, t - tbase);
        const AxisPlan &ap = S.ax[XPASS ? 0 : 1];
        cx<T> *in = reinterpret_cast<cx<T> *>(in0 + (size_t)cur * bstride);
        const bool ok = mbar_wait(&bar[cur], (ph >> cur) & 1u);
        ph ^= 1u << cur;
        pending &= ~(1u << cur);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) {
                atomicExch(err, 1);
                for (int k = 0; k < nin; ++k)     // let the copies in flight land
                    if ((pending >> k) & 1u) mbar_wait(&bar[k], (ph >> k) & 1u);
            }
            __syncthreads();
            return;
        }
        const int split = sizeof(T) == 4 ? (XPASS ? S.sx1 : S.sy1) : 0;
        cx<T> *R;
        if (split) {
            fft_ip_xy_auto<INV>(in, ap.n, g.L, g.ldr, tw);
            R = in;
        } else {
            R = fft_auto<INV>(in, work, ap, g.L, g.ldr, tw);
        }
        // store the rows back (16-byte vectors), walking (row, e) without division
        cx<T> *spec = reinterpret_cast<cx<T> *>(S.spec) + g.g0;
        if (VDWGB_OK(g.outer >= 0 && g.outer < (XPASS ? S.ny : S.nx) && g.kz0 >= 0 && g.wt >= 1, S.err)) {
            constexpr int PER = 16 / (int)sizeof(cx<T>);   // complex values per vector
            const int h = g.L / PER;                         // L = 20 W: even
            const int de = blockDim.x % h, dr = blockDim.x / h;
            int e = threadIdx.x % h, r = threadIdx.x / h;
            for (; r < g.nrows;) {
                const float4 v = *reinterpret_cast<const float4 *>(R + (size_t)r * g.ldr + PER * e);
                *reinterpret_cast<float4 *>(spec + r * g.rowstride + PER * e) = v;
                e += de;
                r += dr;
                if (e >= h) {
                    e -= h;
                    ++r;
                }
            }
        }
        fence_proxy_async();   // this tile's generic accesses before the next bulk writes
        __syncthreads();
        if (nin == 1) {
            const int tn = t + gridDim.x;
            if (tn < total) {
                if (threadIdx.x < 32) xy_issue<T, XPASS>(sys, prefix, nsys, tn, in, &bar[0], &sS, cur_sys, tbase);
                pending |= 1u;
            }
        }
        cur = cur + 1 == nin ? 0 : cur + 1;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < nin; ++k) mbar_inval(&bar[k]);
}

// ---------------------------------------------------------------------------
// Kernel contraction and energy (procedure step 3): for every half-spectrum
// k-point F_a(k) = sum_b phi_ab(|k|) theta_b(k), written over theta, and the
// energy increment w_k sum_a Re(theta_a^* F_a).  The k-points of a system
// are sorted by kernel-table interval; a chunk (<= 256 k-points, one per
// thread) covers a few consecutive intervals, whose rows [interval][pair]
// are one contiguous block staged in shared memory by one bulk copy.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_contract(const SysDev *__restrict__ sys, const int *__restrict__ prefix,
                                                     int nsys, int total, int maxspan,
                                                     const typename KTab<T>::V *__restrict__ tab,
                                                     int *__restrict__ err) {
    using V = typename KTab<T>::V;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem);
    V *rows = reinterpret_cast<V *>(smem + 32);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned ph = 0u;
    const T inv_dk = (T)(RMAX / (2.0 * 3.14159265358979323846));
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int si = find_sys(prefix, nsys, t);
        const SysDev &S = sys[si];
        const int lt = t - prefix[si];
        int4 c = S.chunks[lt];           // first, count, first interval, intervals
        if (!VDWGB_OK(c.x >= 0 && c.y >= 0 && c.y <= (int)blockDim.x &&
                          (size_t)c.x + c.y <= (size_t)S.nx * S.ny * S.nzh &&
                          (c.w == 0 || (c.z >= 0 && c.z + min(c.w, maxspan) <= NK - 1)),
                      S.err))
            c = make_int4(0, 0, 0, 0);   // checked build: an empty chunk
        const int span = min(c.w, maxspan);
        if (span > 0 && threadIdx.x == 0) {
            const unsigned bytes = (unsigned)((size_t)span * NPAIR * sizeof(V));
            fence_proxy_async();
            mbar_expect_tx(&bar[0], bytes);
            bulk_g2s(rows, tab + (size_t)c.z * NPAIR, bytes, &bar[0]);
        }
        // this thread's k-point: index, theta_a(k)
        const bool have = threadIdx.x < c.y;
        unsigned idx = 0;
        cx<T> th[NQ];
        cx<T> *v = nullptr;
        if (have) {
            idx = S.kidx[c.x + threadIdx.x];
            v = reinterpret_cast<cx<T> *>(S.spec) + (size_t)idx * NQ;
            if (sizeof(cx<T>) == 8) {   // 160-byte record, 16-byte aligned: ten 16-byte loads
                const float4 *v4 = reinterpret_cast<const float4 *>(v);
#pragma unroll
                for (int a = 0; a < NQ / 2; ++a) {
                    const float4 q = v4[a];
                    th[2 * a] = cx<T>{(T)q.x, (T)q.y};
                    th[2 * a + 1] = cx<T>{(T)q.z, (T)q.w};
                }
            } else {
#pragma unroll
                for (int a = 0; a < NQ; ++a) th[a] = v[a];
            }
        }
        if (span > 0) {
            const bool ok = mbar_wait(&bar[0], ph);
            ph ^= 1u;
            if (!__syncthreads_and(ok)) {
                if (threadIdx.x == 0) atomicExch(err, 1);
                return;
            }
        }
        double eacc = 0.0;
        if (have) {
            const int nx = S.nx, ny = S.ny, nz = S.nz, nzh = S.nzh, nyg = S.nyg;
            const int kz = (int)(idx % (unsigned)nzh);
            const int rest = (int)(idx / (unsigned)nzh);
            const int y = S.yoff + rest % ny, x = rest / ny;
            const int mx = fold(x, nx), my = fold(y, nyg);
            const bool nyq_x = (nx % 2 == 0) && (x == nx / 2);
            const bool nyq_y = (nyg % 2 == 0) && (y == nyg / 2);
            const bool nyq_z = (nz % 2 == 0) && (kz == nz / 2);
            const int mz = nyq_z ? -kz : kz;
            const T fx = (T)mx, fy = (T)my, fz = (T)mz;
            const T cxv = nyq_x ? (T)0 : fx, cyv = nyq_y ? (T)0 : fy, czv = nyq_z ? (T)0 : fz;
            T k2 = (T)S.g[0] * fx * fx + (T)S.g[1] * fy * fy + (T)S.g[2] * fz * fz +
                   (T)2 * ((T)S.g[3] * cxv * cyv + (T)S.g[4] * cxv * czv + (T)S.g[5] * cyv * czv);
            k2 = k2 > (T)0 ? k2 : (T)0;
            const T xk = sqrt(k2) * inv_dk;
            const int j = (int)xk;
            const T tt = xk - (T)j;
            cx<T> F[NQ];
#pragma unroll
            for (int a = 0; a < NQ; ++a) F[a] = cx<T>{(T)0, (T)0};
            if (j < NK - 1) {
                // the interval's row: staged in shared memory, else (rounding at a
                // chunk edge) read from the global table
                const bool staged = span > 0 && j >= c.z && j < c.z + span;
                const V *row = staged ? rows + (size_t)(j - c.z) * NPAIR : tab + (size_t)j * NPAIR;
                int pidx = 0;
#pragma unroll
                for (int a = 0; a < NQ; ++a) {
#pragma unroll
                    for (int b = a; b < NQ; ++b) {
                        const V cf = staged ? ld_row(row + pidx) : ld_tab(row + pidx);
                        const T phi = cf.x + tt * (cf.y + tt * (cf.z + tt * cf.w));
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
            const T weight = (kz == 0 || nyq_z) ? (T)1 : (T)2;
            eacc = (double)(weight * e);
            if (sizeof(cx<T>) == 8) {
                float4 *v4 = reinterpret_cast<float4 *>(v);
#pragma unroll
                for (int a = 0; a < NQ / 2; ++a)
                    v4[a] = make_float4((float)F[2 * a].x, (float)F[2 * a].y, (float)F[2 * a + 1].x, (float)F[2 * a + 1].y);
            } else {
#pragma unroll
                for (int a = 0; a < NQ; ++a) v[a] = F[a];
            }
        }
        const double es = block_sum<T>(eacc, red);
        if (threadIdx.x == 0) S.epart[lt] = es;
        fence_proxy_async();
        __syncthreads();   // rows free for the next chunk's copy
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_inval(&bar[0]);
}

// ---------------------------------------------------------------------------
// FP32-mixed contraction (procedure step 3, as k_contract).  One producer
// warp and C32_CWARPS consumer warps per block, one block per SM.  The
// producer stages the block's chunks into a ring of C32_RING slots: for each
// chunk a small descriptor (the system's grid and metric, the chunk record),
// its k-point indices and one bulk copy of its kernel-table rows.  It reads
// the chunk records of its next 32 chunks at once (one per lane) and a
// chunk's indices before the chunk's slot is free.  Each consumer thread owns
// one k-point of a chunk and fetches that k-point's 20 theta values (one
// 160-byte record) itself, with ten 16-byte cp.async copies into its own
// record slot, one chunk ahead: the copies of chunk i + 1 are in flight while
// chunk i is computed, and no thread waits for another thread's copies.
// Records sit 176 bytes apart in shared memory, so a warp's 16-byte loads of
// its records are free of bank conflicts.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_arrive_local(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int C32_THREADS = 32 * (1 + C32_CWARPS);           // producer warp first, then the consumers
static_assert(CHUNK32 == 32 * C32_CWARPS, "one k-point per consumer thread");
constexpr int C32_KPL = CHUNK32 / 32;                        // indices per producer lane and chunk
constexpr int C32_RING = 3;                                  // staged chunks (descriptor, indices, rows)
constexpr int C32_RSTRIDE = 11;                              // float4 per record slot (10 used)

// What the consumers need of a chunk: its system's grid and metric, output
// pointers, and the chunk record.
struct __align__(16) C32Desc {
    int nx, ny, nz, nzh, sx1, sy1;
    int count;       // k-points in the chunk
    int first;       // first kernel-table interval of the chunk
    int span;        // staged intervals (0: the chunk lies beyond the table)
    int lt;          // chunk index within its system (energy partials)
    int nepart;      // energy partials of the system
    int yoff, nyg;   // y positions of this system within a global y axis (slabs)
    float gf[6];
    float4 *spec;
    double *epart;
};

__host__ __device__ inline size_t c32_off_desc() { return 64; }
__host__ __device__ inline size_t c32_off_idx() { return c32_off_desc() + C32_RING * sizeof(C32Desc); }
__host__ __device__ inline size_t c32_off_rec() {
    return (c32_off_idx() + (size_t)C32_RING * CHUNK32 * sizeof(unsigned) + 127) / 128 * 128;
}
__host__ __device__ inline size_t c32_off_rows() {
    return c32_off_rec() + 2 * (size_t)CHUNK32 * C32_RSTRIDE * sizeof(float4);
}
__host__ __device__ inline size_t c32_smem_bytes() {
    return c32_off_rows() + (size_t)C32_RING * SPAN32 * NPAIR * sizeof(float4);
}

// |k| of half-spectrum index idx (positions of the x / y passes mapped to
// frequencies, Nyquist planes with the convention of the FP64 path) as table
// interval j and offset tt in [0, 1), exactly as the host sorted it; weight
// 1 on the kz = 0 and Nyquist planes, 2 elsewhere (the other half of the
// spectrum)
__device__ __forceinline__ void c32_kpoint(const C32Desc &D, unsigned idx, int &j, float &tt, float &weight) {
    const int nx = D.nx, ny = D.ny, nz = D.nz, nzh = D.nzh;
    const int kz = (int)(idx % (unsigned)nzh);
    const int rest = (int)(idx / (unsigned)nzh);
    const int nyg = D.nyg;
    const int y = axis_freq(D.yoff + rest % ny, nyg, D.sy1), x = axis_freq(rest / ny, nx, D.sx1);
    const bool nyq_z = (nz % 2 == 0) && (kz == nz / 2);
    kpoint_interval32(D.gf, fold(x, nx), fold(y, nyg), nyq_z ? -kz : kz, (nx % 2 == 0) && (x == nx / 2),
                      (nyg % 2 == 0) && (y == nyg / 2), nyq_z, j, tt);
    weight = (kz == 0 || nyq_z) ? 1.f : 2.f;
}

// consumer thread k: wait (bounded) for chunk i's slot b, then start the ten
// 16-byte copies of its record of that chunk into record buffer rb (one
// commit group); its index into idx.  False if the wait ran out.
__device__ __forceinline__ bool c32_fetch(int i, int b, int rb, int k, int lane, unsigned long long *full,
                                          const C32Desc *desc, const unsigned *sidx, float4 *srec, int *err,
                                          int *s_failed, unsigned &idx) {
    const bool ok = !*(volatile int *)s_failed && mbar_wait(&full[b], (unsigned)((i / C32_RING) & 1));
    if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) {
            atomicExch(err, 1);
            *s_failed = 1;
        }
        return false;
    }
    const C32Desc &D = desc[b];
    if (k < D.count) {
        idx = sidx[b * CHUNK32 + k];
        if (!VDWGB_OK(idx < (unsigned)(D.nx * D.ny * D.nzh), err)) idx = 0;   // checked build
        const float4 *src = D.spec + (size_t)idx * 10;
        float4 *dst = srec + ((size_t)rb * CHUNK32 + k) * C32_RSTRIDE;
#pragma unroll
        for (int a = 0; a < 10; ++a) cp_async16(dst + a, src + a);
    }
    cp_async_commit();
    return true;
}

__global__ void __launch_bounds__(C32_THREADS, 1) k_contract32(const SysDev *__restrict__ sys, const int *__restrict__ prefix,
                                                             int nsys, int total, const float4 *__restrict__ tab,
                                                             int *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *full = reinterpret_cast<unsigned long long *>(smem);   // [C32_RING]
    unsigned long long *empty = full + C32_RING;                             // [C32_RING]
    C32Desc *desc = reinterpret_cast<C32Desc *>(smem + c32_off_desc());
    unsigned *sidx = reinterpret_cast<unsigned *>(smem + c32_off_idx());
    float4 *srec = reinterpret_cast<float4 *>(smem + c32_off_rec());
    float4 *rows = reinterpret_cast<float4 *>(smem + c32_off_rows());
    __shared__ int s_failed;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_failed = 0;
        for (int r = 0; r < C32_RING; ++r) {
            mbar_init(&full[r], 1);
            mbar_init(&empty[r], C32_CWARPS);
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        // ---- producer warp: descriptors, indices and table rows, C32_RING - 1 chunks ahead
        int4 cl = make_int4(0, 0, 0, 0);   // this lane's chunk record among the next 32 chunks
        int sl = 0, ltl = 0;
        int psi = -1;                      // system of the cached fields below
        C32Desc d;
        const unsigned *gkidx = nullptr;
        unsigned kn[C32_KPL];
        int issued = 0;
        for (int t = blockIdx.x, i = 0, b = 0; t < total; t += gridDim.x, ++i, b = b + 1 == C32_RING ? 0 : b + 1) {
            if ((i & 31) == 0) {
                const int tl = t + lane * gridDim.x;
                if (tl < total) {
                    sl = find_sys(prefix, nsys, tl);
                    ltl = tl - prefix[sl];
                    cl = sys[sl].chunks[ltl];
                }
            }
            const int src = i & 31;
            const int s = __shfl_sync(0xffffffffu, sl, src);
            const int lt = __shfl_sync(0xffffffffu, ltl, src);
            const int cx = __shfl_sync(0xffffffffu, cl.x, src);
            int cy = __shfl_sync(0xffffffffu, cl.y, src);
            const int cz = __shfl_sync(0xffffffffu, cl.z, src);
            int cwv = __shfl_sync(0xffffffffu, cl.w, src);
            if (s != psi) {                // every lane keeps the system's fields
                const SysDev &S = sys[s];
                d.nx = S.nx;
                d.ny = S.ny;
                d.nz = S.nz;
                d.nzh = S.nzh;
                d.sx1 = S.sx1;
                d.sy1 = S.sy1;
#pragma unroll
                for (int q = 0; q < 6; ++q) d.gf[q] = S.gf[q];
                d.spec = reinterpret_cast<float4 *>(S.spec);
                d.epart = S.epart;
                d.nepart = S.nepart;
                d.yoff = S.yoff;
                d.nyg = S.nyg;
                gkidx = S.kidx;
                psi = s;
            }
            // checked build: a chunk record outside the system's k-points or
            // the table is staged as an empty chunk
            if (!VDWGB_OK(cx >= 0 && cy >= 1 && cy <= CHUNK32 &&
                              (size_t)cx + cy <= (size_t)d.nx * d.ny * d.nzh && lt >= 0 &&
                              (cwv == 0 || (cz >= 0 && cz + min(cwv, SPAN32) <= NK - 1)),
                          err)) {
                cy = 0;
                cwv = 0;
            }
            // the chunk's indices into registers (coalesced) before its slot is free
#pragma unroll
            for (int r = 0; r < C32_KPL; ++r) {
                const int k = lane + 32 * r;
                kn[r] = k < cy ? gkidx[cx + k] : 0u;
            }
            if (i >= C32_RING) {
                // slot b released by every consumer warp (its previous use, chunk i - C32_RING)
                const bool ok = mbar_wait(&empty[b], (unsigned)(((i / C32_RING) - 1) & 1));
                if (!__all_sync(0xffffffffu, ok) || *(volatile int *)&s_failed) {
                    if (lane == 0) {
                        atomicExch(err, 1);
                        s_failed = 1;
                    }
                    break;
                }
            }
            const int span = min(cwv, SPAN32);
            // descriptor and indices (generic stores), published to the
            // consumers by lane 0's arrive on full[b] after the warp barrier
#pragma unroll
            for (int r = 0; r < C32_KPL; ++r) {
                const int k = lane + 32 * r;
                if (k < cy) sidx[b * CHUNK32 + k] = kn[r];
            }
            if (lane == 0) {
                d.count = cy;
                d.first = cz;
                d.span = span;
                d.lt = lt;
                desc[b] = d;
            }
            __syncwarp();
            if (lane == 0) {
                fence_proxy_async();
                mbar_expect_tx(&full[b], (unsigned)(span * NPAIR * (int)sizeof(float4)));
                if (span > 0)
                    bulk_g2s(rows + (size_t)b * SPAN32 * NPAIR, tab + (size_t)cz * NPAIR,
                             (unsigned)(span * NPAIR * sizeof(float4)), &full[b]);
            }
            issued = i + 1;
        }
        // every copy issued has landed before the block exits (the last use of each slot)
        if (lane == 0)
            for (int i = issued - C32_RING > 0 ? issued - C32_RING : 0; i < issued; ++i)
                mbar_wait(&full[i % C32_RING], (unsigned)((i / C32_RING) & 1));
    } else {
        // ---- consumer warps: one k-point per thread
        const int cw = (threadIdx.x >> 5) - 1;
        const int k = threadIdx.x - 32;
        unsigned idx = 0;
        bool running = blockIdx.x < total &&
                       c32_fetch(0, 0, 0, k, lane, full, desc, sidx, srec, err, &s_failed, idx);
        for (int t = blockIdx.x, i = 0, b = 0; running && t < total;
             t += gridDim.x, ++i, b = b + 1 == C32_RING ? 0 : b + 1) {
            const unsigned idx_c = idx;
            // the next chunk's record copies, in flight while this chunk is computed
            const bool more = t + gridDim.x < total;
            if (more) {
                const int bn = b + 1 == C32_RING ? 0 : b + 1;
                running = c32_fetch(i + 1, bn, (i + 1) & 1, k, lane, full, desc, sidx, srec, err, &s_failed, idx);
                cp_async_wait<1>();                  // this thread's copies of chunk i have landed
            } else {
                cp_async_wait<0>();
            }
            const C32Desc &D = desc[b];
            double ed = 0.0;
            if (k < D.count) {
                int j;
                float tt, w;
                c32_kpoint(D, idx_c, j, tt, w);
                f2_t th[NQ], F[NQ];
                load_rec_f2(srec + ((size_t)(i & 1) * CHUNK32 + k) * C32_RSTRIDE, th);
#pragma unroll
                for (int a = 0; a < NQ; ++a) F[a] = 0ull;
                // the interval's row is staged: the host sorted this k-point into
                // the chunk with the same FP32 decision (j = NK - 1: beyond the
                // table).  A row outside the staged range would break that
                // invariant: skipped and reported (status 2), never read.
                if (j < NK - 1) {
                    const int r = j - D.first;
                    if (r >= 0 && r < D.span)
                        contract_row<false>(rows + ((size_t)b * SPAN32 + r) * NPAIR, tt, th, F);
                    else
                        atomicExch(err, 2);
                }
                ed = f2d_bits(w * energy_f2(th, F));
                store_rec_f2(D.spec + (size_t)idx_c * 10, F);
            }
            // the warp's k-point energies widened exactly (integer pipe) and
            // summed in FP64: five FP64 additions per warp and chunk
            for (int o = 16; o > 0; o >>= 1) ed += __shfl_down_sync(0xffffffffu, ed, o);
            if (lane == 0 && VDWGB_OK(D.lt * C32_CWARPS + cw < D.nepart, err))
                D.epart[(size_t)D.lt * C32_CWARPS + cw] = ed;
            __syncwarp();                        // the warp's reads of slot b are done
            if (lane == 0) mbar_arrive_local(&empty[b]);
        }
        cp_async_wait<0>();                      // no copy of this thread is in flight at exit
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int r = 0; r < C32_RING; ++r) {
            mbar_inval(&full[r]);
            mbar_inval(&empty[r]);
        }
}

// ---------------------------------------------------------------------------
// z-inverse: complex-to-real along z, then the potential.  A tile is LZi
// consecutive (x, y) lines; their half spectra and point records are one
// contiguous range each, fetched by two bulk copies into a double-buffered
// stage while the previous tile is transformed.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void zinv_issue(const SysDev *__restrict__ sys, const int *__restrict__ prefix, int nsys,
                                           int t, cx<T> *ibuf, Rec<T> *rbuf, unsigned long long *bar,
                                           const SysDev *cached = nullptr, int cached_si = -1, int cached_base = 0) {
    const int si = advance_sys(prefix, nsys, t, cached_si);
    const bool hit = cached && si == cached_si;
    const SysDev &S = hit ? *cached : sys[si];
    const int lt = t - (hit ? cached_base : prefix[si]);
    const int l0 = lt * S.LZi;
    const int nl = min(S.LZi, S.nx * S.ny - l0);
    if (!VDWGB_OK(lt >= 0 && l0 >= 0 && nl >= 1, S.err)) {
        mbar_expect_tx(bar, 0u);                 // complete the phase without copies
        return;
    }
    const unsigned sb = (unsigned)((size_t)nl * S.nzh * NQ * sizeof(cx<T>));
    const unsigned rb = (unsigned)((size_t)nl * S.nz * sizeof(Rec<T>));
    fence_proxy_async();
    mbar_expect_tx(bar, sb + rb);
    bulk_g2s(ibuf, reinterpret_cast<const cx<T> *>(S.spec) + (size_t)l0 * S.nzh * NQ, sb, bar);
    bulk_g2s(rbuf, reinterpret_cast<const Rec<T> *>(S.rec) + (size_t)l0 * S.nz, rb, bar);
}

// Pack the staged (or global) half spectra of nl z-lines into complex
// lines of the transform buffer a ([z][ld], line li * 10 + c):
// Z_c[kz] = X_2c[kz] + i X_2c+1[kz] and, for the mirror, Z_c[nz - kz] =
// conj(X_2c[kz]) + i conj(X_2c+1[kz]); the imaginary parts of the kz = 0 and
// Nyquist bins are dropped (complex-to-real semantics).  One thread handles
// half h (c = 5h .. 5h + 4) of one (line, kz).  No barrier at the end.
template <typename T>
__device__ __forceinline__ void zinv_pack(cx<T> *a, const cx<T> *spec, int nl, int nz, int nzh, int ld) {
    const bool even = (nz % 2) == 0;
    const int half = threadIdx.x & 1;
    const int step = blockDim.x >> 1;
    const int dk = step % nzh, dli = step / nzh;
    int kz = (threadIdx.x >> 1) % nzh, li = (threadIdx.x >> 1) / nzh;
    for (; li < nl;) {
        const cx<T> *in = spec + ((size_t)li * nzh + kz) * NQ + 10 * half;
        const int km = nz - kz;
        const bool mirror = kz > 0 && km >= nzh;
        const bool realbin = kz == 0 || (even && kz == nz / 2);
        cx<T> *o1 = a + (size_t)kz * ld + li * 10 + 5 * half;
        cx<T> *o2 = a + (size_t)(mirror ? km : 0) * ld + li * 10 + 5 * half;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            cx<T> x0, x1;
            if constexpr (sizeof(T) == 4) {
                const float4 v = *reinterpret_cast<const float4 *>(in + 2 * c);
                x0 = cx<T>{v.x, v.y};
                x1 = cx<T>{v.z, v.w};
            } else {
                x0 = in[2 * c];
                x1 = in[2 * c + 1];
            }
            if (realbin) {
                x0.y = (T)0;
                x1.y = (T)0;
            }
            o1[c] = cx<T>{x0.x - x1.y, x0.y + x1.x};
            if (mirror) o2[c] = cx<T>{x0.x + x1.y, x1.x - x0.y};
        }
        kz += dk;
        li += dli;
        if (kz >= nzh) {
            kz -= nzh;
            ++li;
        }
    }
}

// Potential of the z-inverse tile's nl lines (Eq. dedn, Eq. dedsigma):
// dE/dtheta_a = dV F_a; dedn = sum_a F_a (p_a + n p_a' dq0/dn), dedsigma =
// sum_a F_a n p_a' dq0/dsigma (the 1/N of the inverse transform folded in).
// R: the transformed lines in shared memory ([z][ld], line li * 10 + c holds
// F_2c + i F_2c+1); rec: the tile's point records (shared or global memory).
// With D_j = sum_a F_a d2_a[j]:
//   sum_a F_a p_a  = A F_j + B F_{j+1} + cA D_j + cB D_{j+1},
//   sum_a F_a p_a' = (F_{j+1} - F_j) / h + dA D_j + dB D_{j+1}.
template <typename T>
__device__ __forceinline__ void zinv_potential(const SysDev &S, const QShared<T> *qs, const cx<T> *R,
                                               const Rec<T> *rec, int l0, int nl, int ld) {
    const int nz = S.nz;
    const size_t p0 = (size_t)l0 * nz;
    const T invN = sizeof(T) == 4 ? (T)S.invNf : (T)S.invN;
    const int dz = blockDim.x % nz, dli = blockDim.x / nz;
    int z = threadIdx.x % nz, li = threadIdx.x / nz;
    double *gdn = S.dedn + p0, *gds = S.dedsigma + p0;
    for (; li < nl;) {
        const int i = li * nz + z;
        const Rec<T> r = rec[i];
        double dn = 0.0, ds = 0.0;
        if (r.j >= 0) {
            const int j = r.j;
            T r0[NQ], r1[NQ];
            d2_rows<T>(j, qs->d2, r0, r1);
            const cx<T> *src = R + (size_t)z * ld + li * 10;
            T D0 = (T)0, D1 = (T)0;
#pragma unroll
            for (int c = 0; c < 10; ++c) {
                const cx<T> v = src[c];
                D0 += v.x * r0[2 * c] + v.y * r0[2 * c + 1];
                D1 += v.x * r1[2 * c] + v.y * r1[2 * c + 1];
            }
            const T *ft = reinterpret_cast<const T *>(src);
            const T Fj = ft[j], Fj1 = ft[j + 1];
            const T hh6 = qs->hh6[j], h6 = qs->h6[j], B = r.B, A = (T)1 - B;
            const T cA = (A * A * A - A) * hh6;
            const T cB = (B * B * B - B) * hh6;
            const T dA = -((T)3 * A * A - (T)1) * h6;
            const T dB = ((T)3 * B * B - (T)1) * h6;
            const T s0 = (A * Fj + B * Fj1 + cA * D0 + cB * D1) * invN;
            const T s1 = ((Fj1 - Fj) * qs->ih[j] + dA * D0 + dB * D1) * invN;
            if (sizeof(T) == 4) {
                dn = f2d_bits((float)(s0 + r.ndqn * s1));
                ds = f2d_bits((float)(r.ndqs * s1));
            } else {
                dn = (double)(s0 + r.ndqn * s1);
                ds = (double)(r.ndqs * s1);
            }
        }
        gdn[i] = dn;
        gds[i] = ds;
        z += dz;
        li += dli;
        if (z >= nz) {
            z -= nz;
            ++li;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) k_zinv(const SysDev *__restrict__ sys, const int *__restrict__ prefix,
                                              int nsys, int total, int nzmax, int inelems, int recelems,
                                              int abelems, int *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem);
    QShared<T> *qs = reinterpret_cast<QShared<T> *>(smem + 16);
    cx<T> *tw = reinterpret_cast<cx<T> *>(smem + 16 + align_up(sizeof(QShared<T>), 16));
    cx<T> *in0 = tw + ((nzmax + 7) & ~7);
    cx<T> *ins[2] = {in0, in0 + inelems};
    Rec<T> *rec0 = reinterpret_cast<Rec<T> *>(in0 + 2 * (size_t)inelems);
    Rec<T> *recs[2] = {rec0, rec0 + recelems};
    cx<T> *bufA = reinterpret_cast<cx<T> *>(rec0 + 2 * (size_t)recelems);
    cx<T> *bufB = bufA + abelems;
    __shared__ SysDev sS;                    // descriptor of the current tile's system
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    load_qshared(qs);
    __syncthreads();
    if (inelems == 0) {
        // direct form (FP32): the first transform pass (or, on axes without
        // an in-place split, the packing of the complex lines) reads the
        // tile's half spectrum straight from global memory (each ten
        // consecutive threads read one k-point's 160 contiguous bytes) and
        // the potential reads the point records from global memory; nothing
        // is staged, so the block needs only its transform buffers and runs
        // at the occupancy its registers allow
        int cur_sys = -1, tbase = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x) {
            const int nsi = advance_sys(prefix, nsys, t, cur_sys);
            if (nsi != cur_sys) {
                __syncthreads();             // readers of the previous descriptor are done
                copy_sys(&sS, &sys[nsi]);
                __syncthreads();
                const cx<T> *twg = reinterpret_cast<const cx<T> *>(sS.tw[2]);
                for (int i = threadIdx.x; i < sS.nz; i += blockDim.x) tw[i] = twg[i];
                __syncthreads();
                cur_sys = nsi;
                tbase = prefix[nsi];
            }
            const SysDev &S = sS;
            const int l0 = (t - tbase) * S.LZi;
            const int nl = min(S.LZi, S.nx * S.ny - l0);
            if (!VDWGB_OK(t >= tbase && nl >= 1, S.err)) continue;   // tile past the system's lines
            {
                // the next tile's half spectrum and point records (same system)
                // into L2 while this tile runs
                const int tn = t + gridDim.x;
                if (tn < total && tn < tbase + S.tiles[3]) {
                    const int l0n = (tn - tbase) * S.LZi;
                    const int nln = min(S.LZi, S.nx * S.ny - l0n);
                    if (nln > 0) {
                        const char *ps = reinterpret_cast<const char *>(S.spec) +
                                         (size_t)l0n * S.nzh * NQ * sizeof(cx<T>);
                        const size_t bs = (size_t)nln * S.nzh * NQ * sizeof(cx<T>);
                        const char *pr = reinterpret_cast<const char *>(S.rec) + (size_t)l0n * S.nz * sizeof(Rec<T>);
                        const size_t br = (size_t)nln * S.nz * sizeof(Rec<T>);
                        for (size_t o = (size_t)threadIdx.x * 128; o < bs; o += (size_t)blockDim.x * 128)
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(ps + o));
                        for (size_t o = (size_t)threadIdx.x * 128; o < br; o += (size_t)blockDim.x * 128)
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(pr + o));
                    }
                }
            }
            const int ld = z_ld(nl);
            const cx<T> *gspec = reinterpret_cast<const cx<T> *>(S.spec) + (size_t)l0 * S.nzh * NQ;
            cx<T> *R = bufA;
            if (sizeof(T) == 4 && S.sz1) {
                fft_ip_inv_packed_auto<T>(bufA, gspec, S.nz, 10 * nl, ld, S.nzh, tw);
            } else {
                zinv_pack<T>(bufA, gspec, nl, S.nz, S.nzh, ld);
                __syncthreads();
                R = fft_auto<true>(bufA, bufB, S.ax[2], 10 * nl, ld, tw);
            }
            zinv_potential<T>(S, qs, R, reinterpret_cast<const Rec<T> *>(S.rec) + (size_t)l0 * S.nz, l0, nl, ld);
            __syncthreads();                 // bufA is rewritten by the next tile
        }
        if (threadIdx.x == 0) {
            mbar_inval(&bar[0]);
            mbar_inval(&bar[1]);
        }
        return;
    }
    unsigned ph[2] = {0u, 0u};
    int t = blockIdx.x;
    if (t < total && threadIdx.x == 0) zinv_issue<T>(sys, prefix, nsys, t, ins[0], recs[0], &bar[0]);
    int cur_sys = -1, tbase = 0;
    for (int it = 0; t < total; ++it, t += gridDim.x) {
        const int cur = it & 1;
        const int tn = t + gridDim.x;
        const int nsi = advance_sys(prefix, nsys, t, cur_sys);
        if (nsi != cur_sys) {
            __syncthreads();                 // readers of the previous descriptor are done
            copy_sys(&sS, &sys[nsi]);
            __syncthreads();
            const cx<T> *twg = reinterpret_cast<const cx<T> *>(sS.tw[2]);
            for (int i = threadIdx.x; i < sS.nz; i += blockDim.x) tw[i] = twg[i];
            cur_sys = nsi;
            tbase = prefix[nsi];
        }
        if (tn < total && threadIdx.x == 0)
            zinv_issue<T>(sys, prefix, nsys, tn, ins[cur ^ 1], recs[cur ^ 1], &bar[cur ^ 1], &sS, cur_sys, tbase);
        const SysDev &S = sS;
        const int lt = t - tbase;
        const int nz = S.nz, nzh = S.nzh;
        const int l0 = lt * S.LZi;
        const int nl = min(S.LZi, S.nx * S.ny - l0);
        const bool tile_ok = VDWGB_OK(lt >= 0 && l0 >= 0 && nl >= 1, S.err);
        const int L = 10 * nl;
        const bool ok = mbar_wait(&bar[cur], ph[cur]);
        ph[cur] ^= 1u;
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicExch(err, 1);
            if (tn < total) mbar_wait(&bar[cur ^ 1], ph[cur ^ 1]);
            return;
        }
        const cx<T> *spec = ins[cur];
        if (!tile_ok) {                      // nothing staged for it (see zinv_issue)
            __syncthreads();
            continue;
        }
        const int ld = z_ld(nl);
        // FP32 with a split: transformed in place, the first pass reading the
        // complex lines straight from the staged half spectrum; other axes:
        // the complex lines packed into the transform buffer first
        // (zinv_pack), then transformed
        const int zs = sizeof(T) == 4 ? S.sz1 : 0;
        if (!zs) zinv_pack<T>(bufA, spec, nl, nz, nzh, ld);
        cx<T> *R;
        if (zs) {
            fft_ip_inv_packed_auto<T>(bufA, spec, nz, L, ld, nzh, tw);
            R = bufA;
        } else {
            __syncthreads();
            R = fft_auto<true>(bufA, bufB, S.ax[2], L, ld, tw);
        }
        zinv_potential<T>(S, qs, R, recs[cur], l0, nl, ld);
        fence_proxy_async();
        __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_inval(&bar[0]);
        mbar_inval(&bar[1]);
    }
}

// ---------------------------------------------------------------------------
// Energy: E = 1/2 (Omega / N^2) sum_k w_k sum_a Re(theta_a^* F_a), partials
// summed in a fixed order with Neumaier compensation (one block per system).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void neumaier_add(double &s, double &c, double v) {
    const double t = s + v;
    c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
    s = t;
}

constexpr int EF_THREADS = 256, EF_BATCH = 16;

// (s, c) += v: Neumaier compensated sum in FP32 (the pair s + c carries the
// sum to about twice FP32 precision)
__device__ __forceinline__ void neumaier_add_f(float &s, float &c, float v) {
    const float t = s + v;
    c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
    s = t;
}

// T = double: FP64 partials, FP64 compensated sums.  T = float: the FP64
// partials (one per chunk and consumer warp: FP64 sums of the warp's FP32
// k-point energies; or one per plane and cluster rank from the plane kernel)
// are split into FP32 pairs and summed as compensated FP32 pairs on the FP32
// pipe (GB300's FP64 pipe runs at 1/64 of the FP32 rate), then widened on
// the integer pipe.
template <typename T>
__global__ void __launch_bounds__(EF_THREADS) k_efinish(const SysDev *__restrict__ sys, int nsys) {
    // one block per system: each thread sums a strided share of the partials,
    // then the (sum, compensation) pairs meet in a fixed tree (shuffles within
    // warps, then across warps): the same order on every run
    __shared__ T rs[EF_THREADS / 32], rc[EF_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int si = blockIdx.x; si < nsys; si += gridDim.x) {
        const SysDev &S = sys[si];
        const int n = S.nepart;
        const double *ep = S.epart;
        T s = 0, c = 0;
        // batches of EF_BATCH strided loads in flight, then their sums in order
        for (int i0 = threadIdx.x; i0 < n; i0 += EF_THREADS * EF_BATCH) {
            double v[EF_BATCH];
#pragma unroll
            for (int u = 0; u < EF_BATCH; ++u) {
                const int i = i0 + u * EF_THREADS;
                v[u] = i < n ? ep[i] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < EF_BATCH; ++u) {
                if constexpr (sizeof(T) == 8) {
                    neumaier_add(s, c, v[u]);
                } else {
                    const dfl d = df_from_bits(v[u]);   // hi + lo: 48 of the partial's bits
                    neumaier_add_f(s, c, d.hi);
                    c += d.lo;
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const T s2 = __shfl_down_sync(0xffffffffu, s, o);
            const T c2 = __shfl_down_sync(0xffffffffu, c, o);
            if constexpr (sizeof(T) == 8) neumaier_add(s, c, s2);
            else neumaier_add_f(s, c, s2);
            c += c2;
        }
        if (lane == 0) {
            rs[w] = s;
            rc[w] = c;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            T ts = rs[0], tc = rc[0];
            for (int k = 1; k < EF_THREADS / 32; ++k) {
                if constexpr (sizeof(T) == 8) neumaier_add(ts, tc, rs[k]);
                else neumaier_add_f(ts, tc, rs[k]);
                tc += rc[k];
            }
            if constexpr (sizeof(T) == 8) *S.energy = S.escale * (ts + tc);
            else *S.energy = S.escale * (f2d_bits(ts) + f2d_bits(tc));
        }
        __syncthreads();
    }
}

// q0, dq0/dn, dq0/dsigma of the chosen form at given points (checks of the
// q0 step on its own).
template <typename T>
__global__ void k_q0(int npts, const double *__restrict__ n, const double *__restrict__ s, double Z,
                     double *__restrict__ q0, double *__restrict__ dqdn, double *__restrict__ dqds) {
    __shared__ Q0Tab tb;
    load_q0tab(&tb);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts) return;
    if (sizeof(T) == 4) {
        const Q0M q = q0_point_df(n[i], s[i], df_from(-Z / 36.0), &tb);
        q0[i] = q.q0;
        dqdn[i] = q.dqdn;
        dqds[i] = q.dqds;
    } else {
        const Q0 q = q0_point(n[i], s[i], Z);
        q0[i] = q.q0;
        dqdn[i] = q.dqdn;
        dqds[i] = q.dqds;
    }
}

cudaError_t launch_q0(int prec, int npts, const double *n, const double *s, double Z, double *q0, double *dqdn,
                      double *dqds) {
    const int blocks = (npts + 255) / 256;
    if (prec == 1) k_q0<float><<<blocks, 256>>>(npts, n, s, Z, q0, dqdn, dqds);
    else k_q0<double><<<blocks, 256>>>(npts, n, s, Z, q0, dqdn, dqds);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// k-point order (plan step): the half-spectrum k-points of a system sorted by
// kernel-table interval j = floor(|k| / dk), stably (equal intervals keep
// index order), for the contraction's chunks.  Each warp owns a range of
// KSORT_RANGE consecutive k-points: k_ksort_hist counts its range's intervals,
// k_ksort_scan turns the counts into each range's first position per
// interval, and k_ksort_scatter walks the range again in index order, 32 at a
// time, placing each k-point at its interval's next position (the rank among
// equal intervals of the same step from a warp match).  The result is the
// order of a sequential stable counting sort.
// ---------------------------------------------------------------------------
// interval of half-spectrum index idx: FP32-mixed as the contraction decides
// it (kpoint_interval32); FP64 from |k| in FP64 with every rounding explicit
template <bool F32>
__device__ __forceinline__ int ksort_bin(const SysDev &S, unsigned idx) {
    const int nx = S.nx, ny = S.ny, nz = S.nz, nzh = S.nzh;
    const int kz = (int)(idx % (unsigned)nzh);
    const int rest = (int)(idx / (unsigned)nzh);
    const int nyg = S.nyg;
    const int x = axis_freq(rest / ny, nx, S.sx1), y = axis_freq(S.yoff + rest % ny, nyg, S.sy1);
    const int mx = fold(x, nx), my = fold(y, nyg);
    const bool qx = (nx % 2 == 0) && (x == nx / 2), qy = (nyg % 2 == 0) && (y == nyg / 2);
    const bool qz = (nz % 2 == 0) && (kz == nz / 2);
    const int mz = qz ? -kz : kz;
    if constexpr (F32) {
        int j;
        float tt;
        kpoint_interval32(S.gf, mx, my, mz, qx, qy, qz, j, tt);
        return j;
    } else {
        const double fx = (double)mx, fy = (double)my, fz = (double)mz;
        const double cx = qx ? 0.0 : fx, cy = qy ? 0.0 : fy, cz = qz ? 0.0 : fz;
        const double diag = __dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(S.g[0], fx), fx), __dmul_rn(__dmul_rn(S.g[1], fy), fy)),
                                      __dmul_rn(__dmul_rn(S.g[2], fz), fz));
        const double cross = __dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(S.g[3], cx), cy), __dmul_rn(__dmul_rn(S.g[4], cx), cz)),
                                       __dmul_rn(__dmul_rn(S.g[5], cy), cz));
        double k2 = __dadd_rn(diag, __dmul_rn(2.0, cross));
        k2 = k2 > 0.0 ? k2 : 0.0;
        const double q = __ddiv_rn(__dsqrt_rn(k2), 2.0 * 3.14159265358979323846 / RMAX);
        return q < (double)(NK - 1) ? (int)q : NK - 1;
    }
}

constexpr int KSORT_WARPS = 8;

template <bool F32>
__global__ void __launch_bounds__(32 * KSORT_WARPS) k_ksort_hist(SysDev S, int nranges, int *__restrict__ hist) {
    __shared__ int h[KSORT_WARPS][NK];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * KSORT_WARPS + w;
    if (r >= nranges) return;              // warps work alone: no block barrier below
    for (int i = lane; i < NK; i += 32) h[w][i] = 0;
    __syncwarp();
    const size_t nk = (size_t)S.nx * S.ny * S.nzh;
    const size_t b0 = (size_t)r * KSORT_RANGE;
    const size_t b1 = b0 + KSORT_RANGE < nk ? b0 + KSORT_RANGE : nk;
    for (size_t i = b0 + lane; i < b1; i += 32) atomicAdd(&h[w][ksort_bin<F32>(S, (unsigned)i)], 1);
    __syncwarp();
    for (int i = lane; i < NK; i += 32) hist[(size_t)r * NK + i] = h[w][i];
}

// one block of NK threads: thread j turns the counts of interval j into
// each range's first position (in place) and writes the interval's total
__global__ void __launch_bounds__(NK) k_ksort_scan(int nranges, int *__restrict__ hist, int *__restrict__ counts) {
    __shared__ int tot[NK], start[NK];
    const int j = threadIdx.x;
    int run = 0;
    for (int r = 0; r < nranges; ++r) {
        const int v = hist[(size_t)r * NK + j];
        hist[(size_t)r * NK + j] = run;
        run += v;
    }
    counts[j] = run;
    tot[j] = run;
    __syncthreads();
    if (j == 0) {
        int s0 = 0;
        for (int q = 0; q < NK; ++q) {
            start[q] = s0;
            s0 += tot[q];
        }
    }
    __syncthreads();
    const int st = start[j];
    for (int r = 0; r < nranges; ++r) hist[(size_t)r * NK + j] += st;
}

template <bool F32>
__global__ void __launch_bounds__(32 * KSORT_WARPS) k_ksort_scatter(SysDev S, int nranges, const int *__restrict__ off,
                                                                  unsigned *__restrict__ kidx) {
    __shared__ int so[KSORT_WARPS][NK];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * KSORT_WARPS + w;
    if (r >= nranges) return;
    for (int i = lane; i < NK; i += 32) so[w][i] = off[(size_t)r * NK + i];
    __syncwarp();
    const size_t nk = (size_t)S.nx * S.ny * S.nzh;
    const size_t b0 = (size_t)r * KSORT_RANGE;
    const size_t b1 = b0 + KSORT_RANGE < nk ? b0 + KSORT_RANGE : nk;
    for (size_t base = b0; base < b1; base += 32) {
        const size_t i = base + lane;
        const bool in = i < b1;
        const unsigned mask = __ballot_sync(0xffffffffu, in);
        if (in) {
            const int j = ksort_bin<F32>(S, (unsigned)i);
            const unsigned peers = __match_any_sync(mask, j);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            kidx[so[w][j] + rank] = (unsigned)i;
            __syncwarp(mask);
            if (lane == __ffs(peers) - 1) so[w][j] += __popc(peers);
        }
        __syncwarp();
    }
}

size_t ksort_scratch_ints(size_t nk) {
    const size_t nranges = (nk + KSORT_RANGE - 1) / KSORT_RANGE;
    return (nranges + 1) * (size_t)NK;
}

cudaError_t launch_ksort(const SysDev &S, bool f32, unsigned *kidx, int *scratch, cudaStream_t st) {
    const size_t nk = (size_t)S.nx * S.ny * S.nzh;
    const int nranges = (int)((nk + KSORT_RANGE - 1) / KSORT_RANGE);
    int *hist = scratch, *counts = scratch + (size_t)nranges * NK;
    const int blocks = (nranges + KSORT_WARPS - 1) / KSORT_WARPS;
    if (f32) k_ksort_hist<true><<<blocks, 32 * KSORT_WARPS, 0, st>>>(S, nranges, hist);
    else k_ksort_hist<false><<<blocks, 32 * KSORT_WARPS, 0, st>>>(S, nranges, hist);
    k_ksort_scan<<<1, NK, 0, st>>>(nranges, hist, counts);
    if (f32) k_ksort_scatter<true><<<blocks, 32 * KSORT_WARPS, 0, st>>>(S, nranges, hist, kidx);
    else k_ksort_scatter<false><<<blocks, 32 * KSORT_WARPS, 0, st>>>(S, nranges, hist, kidx);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Slab decomposition exchange layout: the spectrum of an x-slab, [xl][y][kz][a]
// with the y axis cut into P ranges of run complex values per x-plane, as
// [xl][d][run]; the send buffer of the all-to-all as [d][xl][run] (each
// destination's part contiguous), which is exactly the layout of the
// destination's ky-slab spectrum [x][yl][kz][a] with x = s nxl + xl.
// ---------------------------------------------------------------------------
__global__ void k_slab_transpose(const float4 *__restrict__ src, float4 *__restrict__ dst, int nxl, int P,
                                 size_t run4, int to_send) {
    const size_t total = (size_t)nxl * P * run4;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t v = i % run4, q = i / run4;
        if (to_send) {                      // i walks the send buffer [d][xl][run]
            const size_t xl = q % nxl, d = q / nxl;
            dst[i] = src[(xl * P + d) * run4 + v];
        } else {                            // i walks the x-slab spectrum [xl][d][run]
            const size_t d = q % P, xl = q / P;
            dst[i] = src[(d * nxl + xl) * run4 + v];
        }
    }
}

cudaError_t launch_slab_transpose(const void *src, void *dst, int nxl, int P, size_t run_bytes, bool to_send,
                                  int sms, cudaStream_t st) {
    const size_t run4 = run_bytes / 16;
    const size_t total = (size_t)nxl * P * run4;
    size_t blocks = (total + 255) / 256;
    if (blocks > (size_t)sms * 8) blocks = (size_t)sms * 8;
    if (blocks < 1) blocks = 1;
    k_slab_transpose<<<(unsigned)blocks, 256, 0, st>>>(static_cast<const float4 *>(src), static_cast<float4 *>(dst),
                                                       nxl, P, run4, to_send ? 1 : 0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
// z passes: one tile buffer when the FP32 transform runs in place, else two
template <typename T>
size_t z_nbuf(int nz) {
    return sizeof(T) == 4 && fft_split(nz) ? 1 : 2;
}
template <typename T>
size_t smem_z(int nz, int LZ) {
    return ((sizeof(QShared<T>) + 15) / 16) * 16 +
           sizeof(cx<T>) * ((size_t)((nz + 1) & ~1) + z_nbuf<T>(nz) * nz * z_ld(LZ));
}
template <typename T>
size_t smem_xy(int n, int W, int nslots) {
    return xy_smem_bytes(n, n * NQ * W, nslots, sizeof(cx<T>));
}

size_t zinv_smem(int prec, int nzmax, int inelems, int recelems, int abelems, int nab);

// z-inverse block: FP32 runs the direct form (no staging: one transform
// buffer with an in-place split, else two), FP64 stages two tiles of input
template <typename T>
size_t smem_zinv(int nz, int LZ) {
    if (sizeof(T) == 4) return zinv_smem(1, nz, 0, 0, nz * z_ld(LZ), fft_split(nz) ? 1 : 2);
    const size_t nzh = nz / 2 + 1;
    return 16 + ((sizeof(QShared<T>) + 15) / 16) * 16 +
           sizeof(cx<T>) * ((size_t)((nz + 7) & ~7) + 2 * (size_t)LZ * nzh * NQ + z_nbuf<T>(nz) * nz * z_ld(LZ)) +
           2 * (size_t)LZ * nz * sizeof(Rec<T>);
}

size_t zinv_smem(int prec, int nzmax, int inelems, int recelems, int abelems, int nab) {
    const bool f = prec == 1;
    const size_t c = f ? sizeof(cx<float>) : sizeof(cx<double>);
    const size_t rs = f ? sizeof(Rec<float>) : sizeof(Rec<double>);
    const size_t qsz = f ? ((sizeof(QShared<float>) + 15) / 16) * 16 : ((sizeof(QShared<double>) + 15) / 16) * 16;
    return 16 + qsz + c * ((size_t)((nzmax + 7) & ~7) + 2 * (size_t)inelems + (size_t)nab * abelems) +
           2 * (size_t)recelems * rs;
}

size_t stage_smem(int stage, int prec, int n, int tile, int nbuf) {
    const bool f = prec == 1;
    switch (stage) {
        case 0: return f ? smem_z<float>(n, tile) : smem_z<double>(n, tile);
        case 3: return f ? smem_zinv<float>(n, tile) : smem_zinv<double>(n, tile);
        default: return f ? smem_xy<float>(n, tile, nbuf) : smem_xy<double>(n, tile, nbuf);
    }
}

static cudaError_t set_smem(const void *fn, size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

template <typename T>
static cudaError_t init_kernels_t(size_t maxsmem) {
    cudaError_t e;
    if ((e = set_smem((const void *)k_zfwd<T>, maxsmem)) != cudaSuccess) return e;
    if ((e = set_smem((const void *)k_xy<T, 0>, maxsmem)) != cudaSuccess) return e;
    if ((e = set_smem((const void *)k_xy<T, 1>, maxsmem)) != cudaSuccess) return e;
    if ((e = set_smem((const void *)k_xy<T, 2>, maxsmem)) != cudaSuccess) return e;
    if ((e = set_smem((const void *)k_xy<T, 3>, maxsmem)) != cudaSuccess) return e;
    if ((e = set_smem((const void *)k_contract<T>, maxsmem - 32 * sizeof(double))) != cudaSuccess) return e;
    if (sizeof(T) == 4 && (e = set_smem((const void *)k_contract32, maxsmem - (C32_THREADS / 32) * sizeof(double))) !=
                              cudaSuccess)
        return e;
    if ((e = set_smem((const void *)k_zinv<T>, maxsmem)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t init_kernels(size_t maxsmem) {
    cudaError_t e = init_kernels_t<float>(maxsmem);
    if (e != cudaSuccess) return e;
    if ((e = init_plane_kernel(maxsmem)) != cudaSuccess) return e;
    return init_kernels_t<double>(maxsmem);
}

template <typename T>
static const void *kind_kernel(int kind) {
    switch (kind) {
        case 0: return (const void *)k_zfwd<T>;
        case 1: return (const void *)k_xy<T, 0>;
        case 2: return (const void *)k_xy<T, 2>;
        case 3: return (const void *)k_zinv<T>;
        default:
            if (sizeof(T) == 4) return (const void *)k_contract32;
            return (const void *)k_contract<T>;
    }
}

int stage_blocks_per_sm(int kind, int prec, size_t smem) {
    const void *fn = prec == 1 ? kind_kernel<float>(kind) : kind_kernel<double>(kind);
    const int threads = (kind == 4 && prec == 1) ? C32_THREADS : 256;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    return n < 1 ? 1 : (n > 8 ? 8 : n);
}

// stage -> tile kind (-1: efinish)
int stage_kind(int stage) {
    static const int kind[NSTAGE] = {0, 5, 1, 2, 4, 2, 1, 3, -1};
    return (stage >= 0 && stage < NSTAGE) ? kind[stage] : -1;
}

template <typename T>
static cudaError_t launch_stage_t(const LaunchSet &ls, int stage, cudaStream_t st) {
    const typename KTab<T>::V *tab = reinterpret_cast<const typename KTab<T>::V *>(ls.table);
    const int kind = stage_kind(stage);
    if (kind >= 0 && ls.total[kind] == 0) return cudaSuccess;     // no tiles of this kind
    switch (stage) {
        case 0:
            k_zfwd<T><<<ls.grid[0], 256, ls.smem[0], st>>>(ls.sys, ls.prefix[0], ls.nsys, ls.total[0]);
            break;
        case 1:
            if (sizeof(T) == 4) return launch_plane(ls, st);
            break;
        case 2:
            k_xy<T, 0><<<ls.grid[1], 256, ls.smem[1], st>>>(ls.sys, ls.prefix[1], ls.nsys, ls.total[1],
                                                             ls.twmax[1], ls.bufelems[1], ls.nbuf[1],
                                                             ls.work[1], ls.err);
            break;
        case 6:
            k_xy<T, 1><<<ls.grid[1], 256, ls.smem[1], st>>>(ls.sys, ls.prefix[1], ls.nsys, ls.total[1],
                                                             ls.twmax[1], ls.bufelems[1], ls.nbuf[1],
                                                             ls.work[1], ls.err);
            break;
        case 3:
            k_xy<T, 2><<<ls.grid[2], 256, ls.smem[2], st>>>(ls.sys, ls.prefix[2], ls.nsys, ls.total[2],
                                                             ls.twmax[2], ls.bufelems[2], ls.nbuf[2],
                                                             ls.work[2], ls.err);
            break;
        case 5:
            k_xy<T, 3><<<ls.grid[2], 256, ls.smem[2], st>>>(ls.sys, ls.prefix[2], ls.nsys, ls.total[2],
                                                             ls.twmax[2], ls.bufelems[2], ls.nbuf[2],
                                                             ls.work[2], ls.err);
            break;
        case 4:
            if (sizeof(T) == 4)
                k_contract32<<<ls.grid[4], C32_THREADS, ls.smem[4], st>>>(ls.sys, ls.prefix[4], ls.nsys, ls.total[4],
                                                                           reinterpret_cast<const float4 *>(tab), ls.err);
            else
                k_contract<T><<<ls.grid[4], 256, ls.smem[4], st>>>(ls.sys, ls.prefix[4], ls.nsys, ls.total[4],
                                                                    ls.maxspan, tab, ls.err);
            break;
        case 7:
            k_zinv<T><<<ls.grid[3], 256, ls.smem[3], st>>>(ls.sys, ls.prefix[3], ls.nsys, ls.total[3], ls.twmax[3],
                                                            ls.bufelems[3], ls.recelems, ls.abelems, ls.err);
            break;
        default:
            k_efinish<T><<<ls.nsys < 1024 ? ls.nsys : 1024, EF_THREADS, 0, st>>>(ls.sys, ls.nsys);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_stage(const LaunchSet &ls, int prec, int stage, cudaStream_t st) {
    if (prec == 1) return launch_stage_t<float>(ls, stage, st);
    return launch_stage_t<double>(ls, stage, st);
}

cudaError_t launch_all(const LaunchSet &ls, int prec, cudaStream_t st, cudaEvent_t *ev) {
    if (ev) cudaEventRecord(ev[0], st);
    for (int k = 0; k < NSTAGE; ++k) {
        const cudaError_t e = prec == 1 ? launch_stage_t<float>(ls, k, st) : launch_stage_t<double>(ls, k, st);
        if (e != cudaSuccess) return e;
        if (ev) cudaEventRecord(ev[k + 1], st);
    }
    return cudaGetLastError();
}

size_t contract_smem(int prec, int maxspan) {
    if (prec == 1) return c32_smem_bytes();
    return 32 + (size_t)maxspan * NPAIR * sizeof(dvec4);
}

const char *stage_name(int i) {
    static const char *names[NSTAGE] = {"zfwd", "plane", "yfwd", "xfwd", "contract", "xinv", "yinv", "zinv",
                                        "efinish"};
    return (i >= 0 && i < NSTAGE) ? names[i] : "";
}


cudaError_t upload_qmesh(const QMeshDev &q) { return cudaMemcpyToSymbol(c_qm, &q, sizeof(QMeshDev)); }

}  // namespace vdwgb
