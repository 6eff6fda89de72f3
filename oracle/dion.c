/*
 * Oracle (test infrastructure only): the Dion et al. kernel phi(d1, d2) by
 * direct double quadrature, in plain FP64 C.
 *
 * The paper takes phi as given ("a precise and universal form that depends
 * only on d1 = q1 r12 and d2 = q2 r12", Sec. after Eq. (Enl)); its definition
 * is Dion et al., PRL 92, 246401 (2004), Eqs. 14-16:
 *
 *   phi(d1,d2) = (2/pi^2) Int_0^inf a^2 da Int_0^inf b^2 db W(a,b) T(nu1(a), nu1(b), nu2(a), nu2(b))
 *   T(w,x,y,z) = 1/2 [1/(w+x) + 1/(y+z)] [1/((w+y)(x+z)) + 1/((w+z)(y+x))]
 *   W(a,b)     = 2 [(3-a^2) b cos b sin a + (3-b^2) a cos a sin b
 *                   + (a^2+b^2-3) sin a sin b - 3 a b cos a cos b] / (a^3 b^3)
 *   nu_i(y)    = y^2 / (2 h(y/d_i)),   h(t) = 1 - exp(-(4 pi/9) t^2)   (h = 1 when d_i = 0)
 *
 * W is evaluated in the algebraically identical form
 *   W(a,b) = 2 [ j0(a) k(b) + j0(b) k(a) - 3 k(a) k(b) ],
 *   j0(x) = sin x / x,  k(x) = (sin x - x cos x) / x^3,
 * with a Taylor series for k at small x, which removes the cancellation of the
 * printed form near a, b -> 0.  A test checks the two forms against each other
 * in multi-precision arithmetic.
 *
 * The caller supplies the quadrature nodes a_i and weights wa_i (weights
 * already include the Jacobian of any variable change).  No tabulation, no
 * interpolation: every requested (d1, d2) is one full double sum.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double PI = 3.14159265358979323846;

/* k(x) = (sin x - x cos x)/x^3 = sum_{n>=1} (-1)^(n+1) 2n x^(2n-2) / (2n+1)! */
static double k_fun(double x) {
    if (fabs(x) < 0.5) {
        double x2 = x * x, term, sum = 0.0, fact = 6.0; /* (2n+1)! for n = 1 */
        double xp = 1.0;
        for (int n = 1; n <= 10; ++n) {
            term = (double)(2 * n) * xp / fact;
            sum += (n % 2 == 1) ? term : -term;
            xp *= x2;
            fact *= (double)(2 * n + 2) * (double)(2 * n + 3);
        }
        return sum;
    }
    return (sin(x) - x * cos(x)) / (x * x * x);
}

static double j0_fun(double x) {
    if (fabs(x) < 1e-4) return 1.0 - x * x / 6.0;
    return sin(x) / x;
}

double oracle_dion_W(double a, double b) {
    double ka = k_fun(a), kb = k_fun(b);
    return 2.0 * (j0_fun(a) * kb + j0_fun(b) * ka - 3.0 * ka * kb);
}

/* nu(y) = y^2/(2 h(y/d)) and its derivative with respect to d */
static void nu_and_dnu(double y, double d, double* nu, double* dnu) {
    if (d <= 0.0) { *nu = 0.5 * y * y; *dnu = 0.0; return; }
    const double gam = 4.0 * PI / 9.0;
    double s = y / d;
    double e = exp(-gam * s * s);
    double h = 1.0 - e;
    if (h <= 0.0) { /* y == 0: nu -> d^2/(2 gamma) */
        *nu = d * d / (2.0 * gam);
        *dnu = d / gam;
        return;
    }
    *nu = y * y / (2.0 * h);
    /* d nu / d d = y^2 gamma s^2 e / (h^2 d) */
    *dnu = y * y * gam * s * s * e / (h * h * d);
}

/*
 * phi[p] = phi(d1[p], d2[p]); if dphi_dd != NULL also the derivative along the
 * ray of fixed d2/d1, d phi / d d with d = sqrt(d1^2 + d2^2).
 */
void oracle_dion_phi(int na, const double* a, const double* wa,
                     int npts, const double* d1, const double* d2,
                     double* phi, double* dphi_dd)
{
    double* K = (double*)malloc(sizeof(double) * (size_t)na * (size_t)na);
    const double pref = 2.0 / (PI * PI);
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < na; ++j)
            K[(size_t)i * na + j] = pref * wa[i] * wa[j] * a[i] * a[i] * a[j] * a[j]
                                  * oracle_dion_W(a[i], a[j]);

#pragma omp parallel
    {
        double* n1 = (double*)malloc(sizeof(double) * 4 * (size_t)na);
        double* n2 = n1 + na;
        double* dn1 = n2 + na;
        double* dn2 = dn1 + na;
#pragma omp for schedule(dynamic, 4)
        for (int p = 0; p < npts; ++p) {
            for (int i = 0; i < na; ++i) {
                nu_and_dnu(a[i], d1[p], &n1[i], &dn1[i]);
                nu_and_dnu(a[i], d2[p], &n2[i], &dn2[i]);
            }
            double sum = 0.0, s1 = 0.0, s2 = 0.0;
            if (dphi_dd == NULL) {
                /* T(w,x,y,z) is unchanged by (a <-> b), i.e. (w,x,y,z) -> (x,w,z,y),
                 * and so is K: sum the upper triangle once, off-diagonal terms twice.
                 * T = 1/2 (w+x+y+z) [(w+z)(y+x) + (w+y)(x+z)]
                 *         / [(w+x)(y+z)(w+y)(x+z)(w+z)(y+x)]                        */
                for (int i = 0; i < na; ++i) {
                    const double w = n1[i], y = n2[i];
                    const double* Ki = K + (size_t)i * na;
                    /* diagonal term j = i: T(w,w,y,y) = 1/(2 w y (w+y)) */
                    double row = Ki[i] / (2.0 * w * y * (w + y));
#pragma omp simd reduction(+:row)
                    for (int j = i + 1; j < na; ++j) {
                        const double x = n1[j], z = n2[j];
                        const double wx = w + x, yz = y + z, wy = w + y, xz = x + z;
                        const double wz = w + z, yx = y + x;
                        const double t = 0.5 * (wx + yz) * (wz * yx + wy * xz)
                                       / (wx * yz * wy * xz * wz * yx);
                        row += 2.0 * Ki[j] * t;
                    }
                    sum += row;
                }
            } else {
                for (int i = 0; i < na; ++i) {
                    const double w = n1[i], y = n2[i];
                    const double* Ki = K + (size_t)i * na;
                    for (int j = 0; j < na; ++j) {
                        const double x = n1[j], z = n2[j];
                        const double iwx = 1.0 / (w + x), iyz = 1.0 / (y + z);
                        const double iwy = 1.0 / (w + y), ixz = 1.0 / (x + z);
                        const double iwz = 1.0 / (w + z), iyx = 1.0 / (y + x);
                        const double S = iwx + iyz;
                        const double P = iwy * ixz + iwz * iyx;
                        sum += Ki[j] * 0.5 * S * P;
                        /* partial derivatives of T = S P / 2 */
                        const double Pw = -iwy * iwy * ixz - iwz * iwz * iyx;
                        const double Px = -iwy * ixz * ixz - iwz * iyx * iyx;
                        const double Py = -iwy * iwy * ixz - iwz * iyx * iyx;
                        const double Pz = -iwy * ixz * ixz - iwz * iwz * iyx;
                        const double Sw = -iwx * iwx, Sy = -iyz * iyz;
                        const double Tw = 0.5 * (Sw * P + S * Pw);
                        const double Tx = 0.5 * (Sw * P + S * Px);
                        const double Ty = 0.5 * (Sy * P + S * Py);
                        const double Tz = 0.5 * (Sy * P + S * Pz);
                        s1 += Ki[j] * (Tw * dn1[i] + Tx * dn1[j]);
                        s2 += Ki[j] * (Ty * dn2[i] + Tz * dn2[j]);
                    }
                }
            }
            phi[p] = sum;
            if (dphi_dd != NULL) {
                double d = sqrt(d1[p] * d1[p] + d2[p] * d2[p]);
                dphi_dd[p] = (d > 0.0) ? (d1[p] * s1 + d2[p] * s2) / d : 0.0;
            }
        }
        free(n1);
    }
    free(K);
}
