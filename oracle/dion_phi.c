/*
 * Oracle (test infrastructure only): the vdW-DF kernel phi(d1, d2) as a plain
 * double sum over a tensor-product quadrature in (a, b).
 *
 * The paper only cites the kernel (Dion et al. 2004, the reference of Eq. 2
 * and of the appendix on q0).  The published form it refers to is
 *
 *   phi(d1, d2) = (2/pi^2) Int_0^inf Int_0^inf a^2 b^2 W(a,b)
 *                  T(nu1(a), nu1(b), nu2(a), nu2(b)) da db
 *   T(w,x,y,z)  = 1/2 [1/(w+x) + 1/(y+z)] [1/((w+y)(x+z)) + 1/((w+z)(y+x))]
 *   nu_i(y)     = y^2 / (2 h(y/d_i)),  h(t) = 1 - exp(-gamma t^2),  gamma = 4 pi / 9
 *
 * The caller (oracle/vdw.py) folds (2/pi^2), the quadrature weights, a^2 b^2
 * and W(a,b) into one symmetric matrix K[i*na + j]; this file only forms the
 * nu values for each (d1, d2) and performs the double sum.  No blocking, no
 * symmetry folding: every (i, j) term is added, in row order.
 *
 * Only tests/, the smoke check and the CPU baseline of the benchmark may load
 * the shared object built from this file.
 */
#include <math.h>

static const double GAMMA_DION = 4.0 * M_PI / 9.0;

/* nu(a) = a^2 / (2 h(a/d)); d == 0 means h == 1 (a/d -> infinity). */
static double nu_of(double a, double d)
{
    if (d == 0.0)
        return 0.5 * a * a;
    double t = a / d;
    double h = -expm1(-GAMMA_DION * t * t); /* 1 - exp(-gamma t^2) without cancellation */
    return 0.5 * a * a / h;
}

static double T_of(double w, double x, double y, double z)
{
    return 0.5 * (1.0 / (w + x) + 1.0 / (y + z)) *
           (1.0 / ((w + y) * (x + z)) + 1.0 / ((w + z) * (y + x)));
}

/*
 * phi for npts pairs (d1[p], d2[p]).
 *   a[na]       quadrature nodes in a (already mapped to (0, a_max))
 *   K[na*na]    (2/pi^2) w_i w_j a_i^2 a_j^2 W(a_i, a_j)
 *   work        2*na doubles per thread are taken from the stack (na <= 4096)
 */
void oracle_phi_batch(long npts, const double *d1, const double *d2,
                      int na, const double *a, const double *K, double *out)
{
    long p;
#pragma omp parallel for schedule(dynamic, 16)
    for (p = 0; p < npts; ++p) {
        double nu1[4096], nu2[4096];
        for (int i = 0; i < na; ++i) {
            nu1[i] = nu_of(a[i], d1[p]);
            nu2[i] = nu_of(a[i], d2[p]);
        }
        double s = 0.0;
        for (int i = 0; i < na; ++i) {
            const double *Ki = K + (long)i * na;
            for (int j = 0; j < na; ++j)
                s += Ki[j] * T_of(nu1[i], nu1[j], nu2[i], nu2[j]);
        }
        out[p] = s;
    }
}

int oracle_num_threads(void)
{
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            n = omp_get_num_threads();
#endif
        }
    }
    return n;
}
