// FP32 kernel contraction of one k-point (procedure step 3 of Sec. 3):
// F_a(k) = sum_b phi_ab(|k|) theta_b(k) over the 210 symmetric pairs a <= b,
// with phi_ab the cubic interpolant of the kernel table in |k| (step 3a).
//
// FP32 table layout (interval-major): row j holds the 210 pairs (a <= b, a
// outer) of interval j as 105 pair-pairs; pair-pair m = pairs 2m and 2m + 1
// is two 16-byte units {c0, c0', c1, c1'} {c2, c2', c3, c3'}, where c_i
// belongs to pair 2m and c_i' to pair 2m + 1 and phi = c0 + c1 t + c2 t^2 +
// c3 t^3 on t in [0, 1).  Two pairs are evaluated with three two-lane FMAs.
//
// theta and F are held as packed (re, im) pairs (64-bit registers), the form
// of a k-point's record in memory (10 x 16 bytes, {re, im} of a = 0..19), so
// each complex multiply-accumulate by the real phi is one two-lane FMA (same
// rounding as two FMAs).
#pragma once
#include "common.cuh"

namespace vdwgb {

typedef unsigned long long f2_t;   // two FP32 lanes (lo = re, hi = im)

constexpr float INV_DK32 = (float)(RMAX / (2.0 * 3.14159265358979323846));   // 1 / table spacing in |k|

// |k| of the signed frequency (mx, my, mz) with the reciprocal metric gf
// (|k|^2 = m^T g m; a Nyquist component enters the diagonal but not the cross
// terms), in FP32, as table interval j (clamped to NK - 1) and offset tt.
// Every rounding is explicit (standalone products, fused multiply-adds and a
// correctly rounded square root), so the host's sort of the k-points into
// intervals and the device's evaluation reach the same j bit for bit.
__host__ __device__ inline void kpoint_interval32(const float *gf, int mx, int my, int mz, bool nyq_x, bool nyq_y,
                                                  bool nyq_z, int &j, float &tt) {
    const float fx = (float)mx, fy = (float)my, fz = (float)mz;
    const float cx = nyq_x ? 0.f : fx, cy = nyq_y ? 0.f : fy, cz = nyq_z ? 0.f : fz;
    const float cross = fmaf(gf[3] * cx, cy, fmaf(gf[4] * cx, cz, (gf[5] * cy) * cz));
    float k2 = fmaf(gf[0] * fx, fx, fmaf(gf[1] * fy, fy, fmaf(gf[2] * fz, fz, 2.f * cross)));
    k2 = k2 > 0.f ? k2 : 0.f;
    const float xk = sqrtf(k2) * INV_DK32;
    j = xk < (float)(NK - 1) ? (int)xk : NK - 1;
    tt = xk - (float)j;
}

// the 20 packed theta_a of a record (generic pointer: shared or global)
__device__ __forceinline__ void load_rec_f2(const float4 *rec, f2_t *v) {
    const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(rec);
#pragma unroll
    for (int m = 0; m < NQ / 2; ++m) {
        const ulonglong2 q = p[m];
        v[2 * m] = q.x;
        v[2 * m + 1] = q.y;
    }
}
__device__ __forceinline__ void store_rec_f2(float4 *rec, const f2_t *v) {
    ulonglong2 *p = reinterpret_cast<ulonglong2 *>(rec);
#pragma unroll
    for (int m = 0; m < NQ / 2; ++m) p[m] = make_ulonglong2(v[2 * m], v[2 * m + 1]);
}
// sum_a Re(theta_a^* F_a) = sum_a (re re + im im)
__device__ __forceinline__ float energy_f2(const f2_t *th, const f2_t *F) {
    f2_t acc = fma_f2(th[0], F[0], 0ull);
#pragma unroll
    for (int a = 1; a < NQ; ++a) acc = fma_f2(th[a], F[a], acc);
    float lo, hi;
    unpack_f2(acc, lo, hi);
    return lo + hi;
}

// F_a += phi_ab(t) theta_b for all pairs of one row.  GLOBAL: the row is
// read from global memory, else from shared memory.
template <bool GLOBAL>
__device__ __forceinline__ void contract_row(const float4 *__restrict__ row, float tt, const f2_t *th, f2_t *F) {
    const ulonglong2 *r2 = reinterpret_cast<const ulonglong2 *>(row);
    const f2_t t2 = pack_f2(tt, tt);
    int pidx = 0;
    float phi_odd = 0.f;   // phi of pair pidx + 1, evaluated with pair pidx
#pragma unroll
    for (int a = 0; a < NQ; ++a) {
#pragma unroll
        for (int bb = a; bb < NQ; ++bb) {
            float phi;
            if ((pidx & 1) == 0) {
                const ulonglong2 lo = GLOBAL ? __ldg(r2 + pidx) : r2[pidx];          // {c0 pair}, {c1 pair}
                const ulonglong2 hi = GLOBAL ? __ldg(r2 + pidx + 1) : r2[pidx + 1];  // {c2 pair}, {c3 pair}
                unpack_f2(fma_f2(fma_f2(fma_f2(hi.y, t2, hi.x), t2, lo.y), t2, lo.x), phi, phi_odd);
            } else {
                phi = phi_odd;
            }
            const f2_t p2 = pack_f2(phi, phi);
            F[a] = fma_f2(p2, th[bb], F[a]);
            if (bb != a) F[bb] = fma_f2(p2, th[a], F[bb]);
            ++pidx;
        }
    }
}

}  // namespace vdwgb
