// Spin-polarised vdW-DF nonlocal correlation (svdW-DF; announced in Sec. 1
// and the outlook of the paper, defined by Thonhauser et al., PRL 115,
// 136402 (2015)).  Everything but q0 is the unpolarised method: theta_a =
// n p_a(q0) with the total density n = n_up + n_dn, the same kernel,
// transforms, contraction and energy (Eq. enlk).  q0 = -(4 pi / 3) eps_xc^0
// (appendix) with spin-scaled exchange, each channel s with k_s =
// (6 pi^2 n_s)^(1/3) and a_s = n_s k_s contributing
//     a_s / n - (Z_ab / 36) sigma_ss / (n a_s),
// and PW92 correlation with its spin interpolation,
//     eps_c = eps_0 + alpha_c f(zeta) / f''(0) (1 - zeta^4) + (eps_1 - eps_0) f(zeta) zeta^4.
//
// On the device:
//   k_spin_q0      n, q0 and dq0/d{n_up, n_dn, sigma_upup, sigma_dndn} in FP64
//                  (FP64 form); k_spin_q0_df the same in double-float
//                  (FP32-mixed form)
//   the pipeline   with the descriptor's q0in set: the z-forward pass takes
//                  q0 as given, the z-inverse pass leaves the two potential
//                  sums S0 = sum_a F_a p_a and S1 = n sum_a F_a p'_a in place
//                  of n and q0
//   k_spin_finish  dE/dn_s = S0 + S1 dq0/dn_s, dE/dsigma_ss = S1 dq0/dsigma_ss
// (Eq. dedn and Eq. dedsigma with the chain rule through the spin q0).
#include <cmath>
#include <mutex>

#include "internal.h"
#include "table.h"
#include "dfmath.cuh"

using namespace vdwgb;

namespace {

struct SpinArgs {
    const double *nu, *nd, *su, *sd;
    double *ntot, *q0, *dq;     // dq: [4][N]
    size_t N;
    double c;                   // Z_ab / 36
    double n_min, q_min, q_cut;
};

// PW92's G(r_s) = -2A (1 + a1 r_s) ln(1 + 1 / (2A (b1 r_s^1/2 + b2 r_s + b3 r_s^3/2 + b4 r_s^2)))
// and dG/dr_s for one parameter set {A, a1, b1, b2, b3, b4}; srs = r_s^1/2,
// isrs = r_s^-1/2
__device__ __forceinline__ void pw92_G(const double *P, double rs, double srs, double isrs, double &g, double &dg) {
    const double A2 = 2.0 * P[0], a1 = P[1], b1 = P[2], b2 = P[3], b3 = P[4], b4 = P[5];
    const double D = A2 * srs * (b1 + srs * (b2 + srs * (b3 + srs * b4)));
    const double dD = A2 * (0.5 * b1 * isrs + b2 + srs * (1.5 * b3 + 2.0 * b4 * srs));
    const double iD = 1.0 / D;
    const double L = log1p(iD);
    const double ar = 1.0 + a1 * rs;
    g = -A2 * ar * L;
    dg = A2 * (ar * dD * iD / (1.0 + D) - a1 * L);
}

__global__ void k_spin_q0(SpinArgs a) {
    // parameter sets: unpolarised (the appendix's), ferromagnetic, -alpha_c (PW92)
    const double P0[6] = {0.031091, 0.2137, 7.5957, 3.5876, 1.6382, 0.49294};
    const double P1[6] = {0.015545, 0.20548, 14.1189, 6.1977, 3.3662, 0.62517};
    const double PA[6] = {0.016887, 0.11125, 10.357, 3.6231, 0.88026, 0.49671};
    const double IFZ20 = 1.0 / 1.709921;                 // 1 / f''(0)
    const double PI = 3.14159265358979323846;
    const double IFDEN = 1.0 / 0.51984209978974632953;   // 1 / (2^(4/3) - 2)
    const double kc = 4.0 * PI / 3.0;
    const double RSK = 1.9191582926775128;               // (9 pi / 4)^(1/3) = r_s k_F
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += (size_t)gridDim.x * blockDim.x) {
        const double nu = a.nu[i] > 0.0 ? a.nu[i] : 0.0, nd = a.nd[i] > 0.0 ? a.nd[i] : 0.0;
        const double su = a.su[i] > 0.0 ? a.su[i] : 0.0, sd = a.sd[i] > 0.0 ? a.sd[i] : 0.0;
        const double n = nu + nd;
        double q0 = a.q_min, d[4] = {0.0, 0.0, 0.0, 0.0};
        if (n > a.n_min) {
            const double inv_n = 1.0 / n;
            // k_F of n and of each channel: k_s = (6 pi^2 n_s)^(1/3), and
            // (1 +- zeta)^(1/3) = (2 n_s / n)^(1/3) = k_s / k_F, r_s = RSK / k_F
            const double kF = cbrt(3.0 * PI * PI * n);
            const double ikF = 1.0 / kF;
            const double kk[2] = {nu > 0.0 ? cbrt(6.0 * PI * PI * nu) : 0.0,
                                  nd > 0.0 ? cbrt(6.0 * PI * PI * nd) : 0.0};
            // exchange of each channel (spin scaling); a channel at or below
            // n_min contributes nothing
            double x = 0.0, own[2] = {0.0, 0.0}, oth[2] = {0.0, 0.0}, sig[2] = {0.0, 0.0};
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const double ns = s ? nd : nu, ss = s ? sd : su;
                if (ns > a.n_min) {
                    const double k = kk[s];
                    const double as = ns * k;
                    const double ia = 1.0 / as;
                    const double gr = a.c * ss * inv_n * ia;        // (Z/36) sigma_ss / (n a_s)
                    x += as * inv_n - gr;
                    own[s] = (4.0 / 3.0) * k * inv_n - as * inv_n * inv_n + gr * (inv_n + (4.0 / 3.0) * k * ia);   // k_s / a_s = 1 / n_s
                    oth[s] = -as * inv_n * inv_n + gr * inv_n;
                    sig[s] = -a.c * inv_n * ia;
                }
            }
            // PW92 correlation at (r_s, zeta); zeta by a correctly rounded
            // division, so that a fully polarised point has zeta = +-1 exactly
            double zeta = (nu - nd) / n;
            zeta = zeta > 1.0 ? 1.0 : (zeta < -1.0 ? -1.0 : zeta);
            const double rs = RSK * ikF, srs = sqrt(rs), isrs = 1.0 / srs;
            double e0, de0, e1, de1, ga, dga;
            pw92_G(P0, rs, srs, isrs, e0, de0);
            pw92_G(P1, rs, srs, isrs, e1, de1);
            pw92_G(PA, rs, srs, isrs, ga, dga);
            const double up = kk[0] * ikF, dn = kk[1] * ikF;
            const double f = ((1.0 + zeta) * up + (1.0 - zeta) * dn - 2.0) * IFDEN;
            const double df = (4.0 / 3.0) * (up - dn) * IFDEN;
            const double z3 = zeta * zeta * zeta, z4 = z3 * zeta;
            const double eps = e0 - ga * f * IFZ20 * (1.0 - z4) + (e1 - e0) * f * z4;
            const double deps_rs = de0 - dga * f * IFZ20 * (1.0 - z4) + (de1 - de0) * f * z4;
            const double deps_z = -ga * IFZ20 * (df * (1.0 - z4) - 4.0 * z3 * f) + (e1 - e0) * (df * z4 + 4.0 * z3 * f);
            const double qraw = x - kc * eps;
            const double common = kc * deps_rs * rs * inv_n * (1.0 / 3.0);
            const double dq_u = own[0] + oth[1] + common - kc * deps_z * (1.0 - zeta) * inv_n;
            const double dq_d = own[1] + oth[0] + common + kc * deps_z * (1.0 + zeta) * inv_n;
            // saturation h_a(x) = a [1 - exp(-sum_{m=1}^{12} (x/a)^m / m)] (appendix)
            const double t = qraw * (1.0 / a.q_cut);
            const double IM[12] = {1.0, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6,
                                   1.0 / 7, 1.0 / 8, 1.0 / 9, 1.0 / 10, 1.0 / 11, 1.0 / 12};
            double S = 0.0, dS = 0.0, tp = 1.0;
#pragma unroll
            for (int m = 0; m < 12; ++m) {
                dS += tp;
                tp *= t;
                S += tp * IM[m];
            }
            const double e = exp(-S);
            const double q = a.q_cut * (1.0 - e);
            if (q >= a.q_min) {
                const double dh = e * dS;
                q0 = q;
                d[0] = dh * dq_u;
                d[1] = dh * dq_d;
                d[2] = dh * sig[0];
                d[3] = dh * sig[1];
            }
        }
        a.ntot[i] = n;
        a.q0[i] = q0;
#pragma unroll
        for (int c = 0; c < 4; ++c) a.dq[c * a.N + i] = d[c];
    }
}

// PW92's G for one parameter set in double-float: gp = -G > 0 and dG/dr_s
__device__ __forceinline__ void pw92_G_df(const double *P, dfl rs, dfl srs, dfl isrs, const float4 *lnt, dfl &gp,
                                          dfl &dg) {
    const double A2 = 2.0 * P[0], a1 = P[1], b1 = P[2], b2 = P[3], b3 = P[4], b4 = P[5];
    dfl poly = df_add_pos(df_mul(DF(b4), srs), DF(b3));
    poly = df_add_pos(df_mul(poly, srs), DF(b2));
    poly = df_add_pos(df_mul(poly, srs), DF(b1));
    const dfl D = df_mul(df_mul(poly, srs), DF(A2));       // 2A (b1 rs^1/2 + b2 rs + b3 rs^3/2 + b4 rs^2)
    dfl dD = df_add_pos(df_mul(DF(0.5 * b1), isrs), DF(b2));
    dD = df_add_pos(dD, df_mul(srs, df_add_pos(DF(1.5 * b3), df_mul(DF(2.0 * b4), srs))));
    dD = df_mul(dD, DF(A2));
    const dfl iD = df_rcp_fast(D);
    const dfl L = df_log1p(iD, lnt);
    const dfl ar = df_add_pos(DF(1.0), df_mul(DF(a1), rs));
    gp = df_mul(df_mul(DF(A2), ar), L);
    dg = df_sub(df_mul(df_mul(DF(A2), ar), df_mul(dD, df_rcp_fast(df_add_pos(D, df_mul(D, D))))),
                df_mul(DF(A2 * a1), L));
}

// The same q0 and derivatives in double-float arithmetic (about 46 bits),
// the FP32-mixed form's counterpart of the FP64 kernel above (the FP64 pipe
// runs at 1/64 of the FP32 rate); the derivatives are rounded to FP32 by
// the saturation slope h'(x), as in the plain form
__global__ void k_spin_q0_df(SpinArgs a) {
    __shared__ float4 lnt[64];
    __shared__ float2 ex2[64];
    load_df_tables(lnt, ex2);
    __syncthreads();
    const double P0[6] = {0.031091, 0.2137, 7.5957, 3.5876, 1.6382, 0.49294};
    const double P1[6] = {0.015545, 0.20548, 14.1189, 6.1977, 3.3662, 0.62517};
    const double PA[6] = {0.016887, 0.11125, 10.357, 3.6231, 0.88026, 0.49671};
    const double PI = 3.14159265358979323846;
    const dfl IFZ20 = DF(1.0 / 1.709921), IFDEN = DF(1.0 / 0.51984209978974632953);
    const dfl KC = DF(4.0 * PI / 3.0);
    const dfl zc = df_from(-a.c);                          // -Z_ab / 36 > 0
    const float qcut = (float)a.q_cut;
    const dfl iqcut = df_from(1.0 / a.q_cut);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += (size_t)gridDim.x * blockDim.x) {
        const double nu = a.nu[i] > 0.0 ? a.nu[i] : 0.0, nd = a.nd[i] > 0.0 ? a.nd[i] : 0.0;
        const double su = a.su[i] > 0.0 ? a.su[i] : 0.0, sd = a.sd[i] > 0.0 ? a.sd[i] : 0.0;
        const double n = nu + nd;
        double q0 = a.q_min, d[4] = {0.0, 0.0, 0.0, 0.0};
        if (n > a.n_min) {
            const dfl nD = df_from_bits(n);
            const dfl inv_n = df_rcp_fast(nD);
            const dfl kF = df_cbrt(df_mul(nD, DF(3.0 * PI * PI)));
            const dfl ikF = df_rcp_fast(kF);
            const double ns2[2] = {nu, nd}, ss2[2] = {su, sd};
            dfl kk[2] = {DF(0.0), DF(0.0)};
            // exchange of each channel (spin scaling); a channel at or below
            // n_min contributes nothing
            dfl x = DF(0.0), own[2] = {DF(0.0), DF(0.0)}, oth[2] = {DF(0.0), DF(0.0)}, sig[2] = {DF(0.0), DF(0.0)};
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const double ns = ns2[s];
                if (ns > 0.0) kk[s] = df_cbrt(df_mul(df_from_bits(ns), DF(6.0 * PI * PI)));
                if (ns > a.n_min) {
                    const dfl nsD = df_from_bits(ns);
                    const dfl as = df_mul(nsD, kk[s]);
                    const dfl ia = df_rcp_fast(as);
                    const dfl gp = df_mul(df_mul(df_mul(zc, df_from_bits(ss2[s])), inv_n), ia);   // -(Z/36) s / (n a)
                    const dfl asn = df_mul(as, inv_n);
                    x = df_add_pos(x, df_add_pos(asn, gp));
                    const dfl asn2 = df_mul(asn, inv_n);
                    const dfl t1 = df_mul(DF(4.0 / 3.0), df_mul(kk[s], inv_n));
                    const dfl t3 = df_mul(gp, df_add_pos(inv_n, df_mul(DF(4.0 / 3.0), df_mul(kk[s], ia))));
                    own[s] = df_sub(df_sub(t1, asn2), t3);
                    oth[s] = df_neg(df_add_pos(asn2, df_mul(gp, inv_n)));
                    sig[s] = df_mul(df_mul(zc, inv_n), ia);
                }
            }
            dfl zeta = df_mul(df_sub(df_from_bits(nu), df_from_bits(nd)), inv_n);
            if (zeta.hi >= 1.f) zeta = DF(1.0);
            if (zeta.hi <= -1.f) zeta = DF(-1.0);
            const dfl rs = df_mul(ikF, DF(1.9191582926775128));   // (9 pi / 4)^(1/3) / k_F
            const dfl srs = df_sqrt(rs);
            const dfl isrs = df_rcp_fast(srs);
            dfl g0, dg0, g1, dg1, gA, dgA;                         // g = -G
            pw92_G_df(P0, rs, srs, isrs, lnt, g0, dg0);
            pw92_G_df(P1, rs, srs, isrs, lnt, g1, dg1);
            pw92_G_df(PA, rs, srs, isrs, lnt, gA, dgA);
            const dfl up = df_mul(kk[0], ikF), dn = df_mul(kk[1], ikF);   // (1 +- zeta)^(1/3)
            const dfl one_p = df_add(DF(1.0), zeta), one_m = df_sub(DF(1.0), zeta);
            const dfl f = df_mul(df_sub(df_add(df_mul(one_p, up), df_mul(one_m, dn)), DF(2.0)), IFDEN);
            const dfl fd = df_mul(df_mul(DF(4.0 / 3.0), df_sub(up, dn)), IFDEN);
            const dfl z3 = df_mul(df_mul(zeta, zeta), zeta), z4 = df_mul(z3, zeta);
            const dfl w1 = df_mul(df_mul(f, IFZ20), df_sub(DF(1.0), z4));   // f (1 - z^4) / f''(0)
            const dfl w2 = df_mul(f, z4);
            // -eps = g0 - gA w1 - (g0 - g1) w2   (G = -g; alpha_c = g_A)
            const dfl g01 = df_sub(g0, g1);
            const dfl meps = df_sub(df_sub(g0, df_mul(gA, w1)), df_mul(g01, w2));
            const dfl deps_rs = df_add(df_sub(dg0, df_mul(dgA, w1)), df_mul(df_sub(dg1, dg0), w2));
            const dfl four_z3f = df_mul(DF(4.0), df_mul(z3, f));
            // deps/dzeta = g_A (fd (1 - z^4) - 4 z^3 f) / f''(0) - (g1 - g0) ... with G = -g:
            // -G_A (...) / f''(0) + (G1 - G0)(fd z^4 + 4 z^3 f) = g_A (...) / f''(0) + (g0 - g1)(...)
            const dfl deps_z = df_add(df_mul(df_mul(gA, IFZ20), df_sub(df_mul(fd, df_sub(DF(1.0), z4)), four_z3f)),
                                      df_mul(g01, df_add(df_mul(fd, z4), four_z3f)));
            const dfl qraw = df_add_pos(x, df_mul(KC, meps));
            const dfl common = df_mul(df_mul(df_mul(KC, deps_rs), rs), df_mul(inv_n, DF(1.0 / 3.0)));
            const dfl zt = df_mul(df_mul(KC, deps_z), inv_n);
            const dfl dq_u = df_sub(df_add(df_add(own[0], oth[1]), common), df_mul(zt, one_m));
            const dfl dq_d = df_add(df_add(df_add(own[1], oth[0]), common), df_mul(zt, one_p));
            float dh = 0.f;
            const dfl q = df_saturate(df_mul(qraw, iqcut), qcut, ex2, dh);
            const double qd = df_to(q);
            if (qd >= a.q_min) {
                q0 = qd;
                d[0] = (double)dh * df_to(dq_u);
                d[1] = (double)dh * df_to(dq_d);
                d[2] = (double)dh * df_to(sig[0]);
                d[3] = (double)dh * df_to(sig[1]);
            }
        }
        a.ntot[i] = n;
        a.q0[i] = q0;
#pragma unroll
        for (int c = 0; c < 4; ++c) a.dq[c * a.N + i] = d[c];
    }
}

__global__ void k_spin_finish(const double *__restrict__ S0, const double *__restrict__ S1,
                              const double *__restrict__ dq, size_t N, double *__restrict__ onu,
                              double *__restrict__ ond, double *__restrict__ osu, double *__restrict__ osd) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const double s0 = S0[i], s1 = S1[i];
        onu[i] = s0 + s1 * dq[i];
        ond[i] = s0 + s1 * dq[N + i];
        osu[i] = s1 * dq[2 * N + i];
        osd[i] = s1 * dq[3 * N + i];
    }
}

const QMeshDev &qmesh() {
    static QMeshDev q;
    static std::once_flag once;
    std::call_once(once, [] { host_qmesh(q); });
    return q;
}

unsigned spin_grid(int device, size_t N) {
    const size_t want = (N + 255) / 256;
    const size_t cap = (size_t)device_sms(device) * 8;
    return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

extern "C" {

int vdwgb_calculate_spin_device(vdwgb_handle h, const double *d_rho_up, const double *d_rho_dn,
                                const double *d_sigma_upup, const double *d_sigma_dndn, double *d_dedrho_up,
                                double *d_dedrho_dn, double *d_dedsigma_upup, double *d_dedsigma_dndn,
                                double *d_energy, void *cuda_stream) {
    if (!h) return fail(VDWGB_EINVAL, "null handle");
    if (!h->inited) return fail(VDWGB_ESTATE, "calculate before init");
    if (!d_rho_up || !d_rho_dn || !d_sigma_upup || !d_sigma_dndn || !d_dedrho_up || !d_dedrho_dn ||
        !d_dedsigma_upup || !d_dedsigma_dndn || !d_energy)
        return fail(VDWGB_EINVAL, "null array");
    if (h->hsys.fused) return fail(VDWGB_ESTATE, "spin-polarised form with the plane kernel");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const size_t N = (size_t)h->nx * h->ny * h->nz;
    if (!h->d_spin) {
        e = device_malloc(reinterpret_cast<void **>(&h->d_spin), 6 * N * sizeof(double));
        if (e != cudaSuccess) return cuda_fail(e, "spin work arrays");
        h->bytes += 6 * N * sizeof(double);
    }
    double *ntot = h->d_spin, *q0 = ntot + N, *dq = q0 + N;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const QMeshDev &qm = qmesh();
    SpinArgs a{d_rho_up, d_rho_dn, d_sigma_upup, d_sigma_dndn, ntot, q0, dq, N, h->hsys.Z / 36.0,
               qm.n_min, qm.q_min, qm.q_cut};
    const unsigned grid = spin_grid(h->device, N);
    if (h->prec == VDWGB_FP32_MIXED) k_spin_q0_df<<<grid, 256, 0, st>>>(a);
    else k_spin_q0<<<grid, 256, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "spin q0");
    // the pipeline reads n and q0 and leaves S0 in n's array, S1 in q0's
    h->hsys.q0in = 1;
    h->last_ptr[0] = nullptr;
    int rc = handle_set_io(h, ntot, q0, ntot, q0, d_energy, st);
    // back to the plain form on the host: the next plain call re-uploads
    h->hsys.q0in = 0;
    h->last_ptr[0] = nullptr;
    if (rc) return rc;
    if ((e = launch_all(h->ls, h->prec, st)) != cudaSuccess) return cuda_fail(e, "launch");
    k_spin_finish<<<grid, 256, 0, st>>>(ntot, q0, dq, N, d_dedrho_up, d_dedrho_dn, d_dedsigma_upup,
                                         d_dedsigma_dndn);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "spin potentials");
    return 0;
}

int vdwgb_calculate_spin(vdwgb_handle h, const double *rho_up, const double *rho_dn, const double *sigma_upup,
                         const double *sigma_dndn, double *dedrho_up, double *dedrho_dn, double *dedsigma_upup,
                         double *dedsigma_dndn, double *energy) {
    if (!h) return fail(VDWGB_EINVAL, "null handle");
    if (!h->inited) return fail(VDWGB_ESTATE, "calculate before init");
    if (!rho_up || !rho_dn || !sigma_upup || !sigma_dndn || !dedrho_up || !dedrho_dn || !dedsigma_upup ||
        !dedsigma_dndn || !energy)
        return fail(VDWGB_EINVAL, "null array");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const size_t N = (size_t)h->nx * h->ny * h->nz;
    if (!h->d_spin_io) {
        e = device_malloc(reinterpret_cast<void **>(&h->d_spin_io), (8 * N + 1) * sizeof(double));
        if (e != cudaSuccess) return cuda_fail(e, "spin staging");
        h->bytes += (8 * N + 1) * sizeof(double);
    }
    double *io = h->d_spin_io;
    const double *hin[4] = {rho_up, rho_dn, sigma_upup, sigma_dndn};
    double *hout[4] = {dedrho_up, dedrho_dn, dedsigma_upup, dedsigma_dndn};
    cudaStream_t st = h->stream;
    for (int c = 0; c < 4 && e == cudaSuccess; ++c)
        e = cudaMemcpyAsync(io + c * N, hin[c], N * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy inputs");
    double *out = io + 4 * N;
    int rc = vdwgb_calculate_spin_device(h, io, io + N, io + 2 * N, io + 3 * N, out, out + N, out + 2 * N,
                                         out + 3 * N, out + 4 * N, st);
    if (rc) return rc;
    for (int c = 0; c < 4 && e == cudaSuccess; ++c)
        e = cudaMemcpyAsync(hout[c], out + c * N, N * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(energy, out + 4 * N, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "copy outputs");
    return vdwgb_device_status(h->device);
}

}  // extern "C"
