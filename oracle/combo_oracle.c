/*
 * combo_oracle.c -- plain, slow FP64 CPU oracle for ComBo FFT homogenization.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests/, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no source, header, table or helper with the CUDA
 * library: it has its own complex FFT (recursive mixed radix, full complex
 * c2c), its own complex derivative symbol, explicit 9x9 complex Green-operator
 * matrices per frequency, dense 9x9 tangents and dense 9x3 D matrices.
 *
 * Paper: "FFT-based homogenization at finite strains using composite boxels
 * (ComBo)", Keshav, Fritzen, Kabel (arXiv 2204.13624).  Citations below name
 * the paper's sections, equations and algorithms.
 *
 * Conventions (Sec. 1.5 "Notation", Eq. (1) vector notation): a 2-tensor F is
 * stored row-major, F[3*i+J] = F_iJ.  A 4-tensor is a 9x9 matrix
 * A[(3i+J)*9 + 3k+L] = A_iJkL.  Fields are component-major: X[c*V + v] with
 * v = x + n1*(y + n2*z), x fastest.  Phase "+" is the inclusion (material
 * index 1), phase "-" the matrix (index 0); the boxel normal N points out of
 * the inclusion into the matrix (Sec. 1.5, Sec. 5.1).
 *
 * Readings of the paper that this file takes (the paper is silent or
 * inconsistent there) are marked READING.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_OK 0
#define ORC_E_INVALID (-1)
#define ORC_E_NOT_CONVERGED (-3)
#define ORC_E_LAMINATE (-4)
#define ORC_E_INADMISSIBLE (-5)
#define ORC_E_NAN (-6)

/* ------------------------------------------------------------------ */
/* 3x3 helpers                                                          */
/* ------------------------------------------------------------------ */
static double det3(const double F[9])
{
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
           F[2] * (F[3] * F[7] - F[4] * F[6]);
}

/* G = F^{-1} via the adjugate. */
static void inv3(const double F[9], double J, double G[9])
{
    G[0] = (F[4] * F[8] - F[5] * F[7]) / J;
    G[1] = (F[2] * F[7] - F[1] * F[8]) / J;
    G[2] = (F[1] * F[5] - F[2] * F[4]) / J;
    G[3] = (F[5] * F[6] - F[3] * F[8]) / J;
    G[4] = (F[0] * F[8] - F[2] * F[6]) / J;
    G[5] = (F[2] * F[3] - F[0] * F[5]) / J;
    G[6] = (F[3] * F[7] - F[4] * F[6]) / J;
    G[7] = (F[1] * F[6] - F[0] * F[7]) / J;
    G[8] = (F[0] * F[4] - F[1] * F[3]) / J;
}

/* Solve the 3x3 system M x = b by Gaussian elimination with partial pivoting. */
static int solve3(const double Min[9], const double b[3], double x[3])
{
    double M[3][4];
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++) M[i][j] = Min[3 * i + j];
        M[i][3] = b[i];
    }
    for (int c = 0; c < 3; c++) {
        int p = c;
        for (int r = c + 1; r < 3; r++)
            if (fabs(M[r][c]) > fabs(M[p][c])) p = r;
        if (M[p][c] == 0.0) return -1;
        if (p != c)
            for (int j = 0; j < 4; j++) {
                double t = M[c][j];
                M[c][j] = M[p][j];
                M[p][j] = t;
            }
        for (int r = c + 1; r < 3; r++) {
            double f = M[r][c] / M[c][c];
            for (int j = c; j < 4; j++) M[r][j] -= f * M[c][j];
        }
    }
    for (int i = 2; i >= 0; i--) {
        double s = M[i][3];
        for (int j = i + 1; j < 3; j++) s -= M[i][j] * x[j];
        x[i] = s / M[i][i];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Compressible Neo-Hookean material, Sec. 6.1:                        */
/*   W = lam/2 (ln J)^2 - mu ln J + mu/2 (tr C - 3),  C = F^T F.         */
/* P = dW/dF = mu F + (lam ln J - mu) F^{-T}                            */
/* A_iJkL = dP_iJ/dF_kL = mu d_ik d_JL + lam G_Ji G_Lk                  */
/*                        + (mu - lam ln J) G_Jk G_Li,    G = F^{-1}.    */
/* ------------------------------------------------------------------ */
double orc_neohooke_energy(const double F[9], double mu, double lam)
{
    double J = det3(F);
    if (!(J > 0.0)) return NAN;
    double trC = 0.0;
    for (int q = 0; q < 9; q++) trC += F[q] * F[q];
    double lnJ = log(J);
    return 0.5 * lam * lnJ * lnJ - mu * lnJ + 0.5 * mu * (trC - 3.0);
}

int orc_neohooke(const double F[9], double mu, double lam, double P[9], double A[81])
{
    double J = det3(F);
    if (!(J > 0.0)) return ORC_E_INADMISSIBLE;
    double G[9];
    inv3(F, J, G);
    double lnJ = log(J);
    for (int i = 0; i < 3; i++)
        for (int Jx = 0; Jx < 3; Jx++) P[3 * i + Jx] = mu * F[3 * i + Jx] + (lam * lnJ - mu) * G[3 * Jx + i];
    if (A) {
        for (int i = 0; i < 3; i++)
            for (int Jx = 0; Jx < 3; Jx++)
                for (int k = 0; k < 3; k++)
                    for (int L = 0; L < 3; L++) {
                        double v = lam * G[3 * Jx + i] * G[3 * L + k] + (mu - lam * lnJ) * G[3 * Jx + k] * G[3 * L + i];
                        if (i == k && Jx == L) v += mu;
                        A[(3 * i + Jx) * 9 + 3 * k + L] = v;
                    }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* ComBo rank-one laminate, Sec. 4.1 and 4.2.                           */
/* ------------------------------------------------------------------ */

/* D matrix of Eq. (Hessian:F): vec(a (x) N) = D a, D_(iJ),k = d_ik N_J.
 * READING: the printed D repeats diag(N1,N2,N3) in every block of three
 * rows, which contradicts the row-major vector notation of Eq. (1); the
 * matrix that maps a to the row-major vector of a (x) N is the one here. */
static void build_D(const double N[3], double D[27])
{
    for (int i = 0; i < 3; i++)
        for (int Jx = 0; Jx < 3; Jx++)
            for (int k = 0; k < 3; k++) D[(3 * i + Jx) * 3 + k] = (i == k) ? N[Jx] : 0.0;
}

/* Delta = D^T M D for a 9x9 M (Eq. (Hessian:F)). */
static void DtMD(const double D[27], const double M[81], double out[9])
{
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double s = 0.0;
            for (int r = 0; r < 9; r++)
                for (int q = 0; q < 9; q++) s += D[r * 3 + a] * M[r * 9 + q] * D[q * 3 + b];
            out[3 * a + b] = s;
        }
}

typedef struct {
    double Fp[9], Fm[9], Pp[9], Pm[9], Ap[81], Am[81];
    double f[3];
    double err, eps;
} lam_state;

/* F(+/-) = Fb +/- (1/c(+/-)) a (x) N (Eq. (Fpm)); material model in both phases
 * (Algorithm 1); traction residual f = (P+ - P-) N (Eq. (tractionbalance)). */
static int lam_eval(const double Fb[9], const double N[3], double cp, double cm, const double mat[4],
                    const double a[3], double tol_rel, double tol_abs, lam_state* s)
{
    for (int i = 0; i < 3; i++)
        for (int Jx = 0; Jx < 3; Jx++) {
            s->Fp[3 * i + Jx] = Fb[3 * i + Jx] + a[i] * N[Jx] / cp;
            s->Fm[3 * i + Jx] = Fb[3 * i + Jx] - a[i] * N[Jx] / cm;
        }
    /* mat = {mu_matrix, lam_matrix, mu_inclusion, lam_inclusion} */
    if (orc_neohooke(s->Fp, mat[2], mat[3], s->Pp, s->Ap)) return ORC_E_LAMINATE;
    if (orc_neohooke(s->Fm, mat[0], mat[1], s->Pm, s->Am)) return ORC_E_LAMINATE;
    double tp = 0.0, tm = 0.0;
    for (int i = 0; i < 3; i++) {
        double ti_p = 0.0, ti_m = 0.0;
        for (int Jx = 0; Jx < 3; Jx++) {
            ti_p += s->Pp[3 * i + Jx] * N[Jx];
            ti_m += s->Pm[3 * i + Jx] * N[Jx];
        }
        s->f[i] = ti_p - ti_m;
        tp += ti_p * ti_p;
        tm += ti_m * ti_m;
    }
    s->err = sqrt(s->f[0] * s->f[0] + s->f[1] * s->f[1] + s->f[2] * s->f[2]);
    double mumax = mat[0] > mat[2] ? mat[0] : mat[2];
    /* READING: the paper leaves the NR tolerance epsilon open (Algorithm 1);
     * we stop at |f| <= tol_rel (|P+ N| + |P- N|) + tol_abs mu_max. */
    s->eps = tol_rel * (sqrt(tp) + sqrt(tm)) + tol_abs * mumax;
    return ORC_OK;
}

/*
 * Laminate evaluation of one composite boxel: Algorithm 1 (Newton-Raphson on
 * the jump vector a) with Algorithm 2 (selective back-projection, Sec. 4.2),
 * then the boxel stress of Eq. (Peff:Seff) and the boxel tangent
 *   A_box = (c+ A+ + c- A-) - dA D Delta^{-1} D^T dA,  dA = A+ - A-.
 * READING: the paper prints "c- A+" in the first bracket of the tangent; the
 * volume average c+ A+ + c- A- (cheat-sheet table, "A_v bar") is used.
 *
 * a_io: in = warm start (used if admissible at Fb, else 0; Algorithm 1 allows
 * any admissible start), out = converged jump.  mat = {mu-, lam-, mu+, lam+}.
 * trace (optional, 4*(max_iter+1) doubles): per iterate k, {beta_k, J+_k,
 * J-_k, |f|_k}.
 */
int orc_laminate(const double Fb[9], const double N[3], double c, const double mat[4], double a_io[3],
                 double tol_rel, double tol_abs, int max_iter, double P[9], double A[81], int* iters_out,
                 int* nbp_out, double* trace)
{
    double cp = c, cm = 1.0 - c;
    if (!(cp > 0.0 && cm > 0.0)) return ORC_E_INVALID;
    double Jb = det3(Fb);
    if (!(Jb > 0.0)) return ORC_E_INADMISSIBLE;
    double G[9];
    inv3(Fb, Jb, G);
    /* m_beta = F^{-T} N / |F^{-T} N|, beta_c(+/-) = -/+ c(+/-) / |F^{-T} N|  (Sec. 4.2) */
    double g[3];
    for (int i = 0; i < 3; i++) g[i] = G[0 * 3 + i] * N[0] + G[1 * 3 + i] * N[1] + G[2 * 3 + i] * N[2];
    double ng = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    double m[3] = {g[0] / ng, g[1] / ng, g[2] / ng};
    double bcp = -cp / ng, bcm = cm / ng;

    double a[3] = {a_io[0], a_io[1], a_io[2]};
    double beta = a[0] * m[0] + a[1] * m[1] + a[2] * m[2];
    if (!(beta > bcp && beta < bcm)) a[0] = a[1] = a[2] = 0.0; /* admissible start (Eq. (matrixlemma)) */

    double D[27];
    build_D(N, D);
    lam_state s;
    int rc = lam_eval(Fb, N, cp, cm, mat, a, tol_rel, tol_abs, &s);
    if (rc) return rc;
    int it = 0, nbp = 0;
    if (trace) {
        trace[0] = a[0] * m[0] + a[1] * m[1] + a[2] * m[2];
        trace[1] = det3(s.Fp);
        trace[2] = det3(s.Fm);
        trace[3] = s.err;
    }
    double M9[81], Delta[9];
    while (s.err > s.eps) {
        if (it >= max_iter) return ORC_E_LAMINATE;
        for (int q = 0; q < 81; q++) M9[q] = s.Ap[q] / cp + s.Am[q] / cm;
        DtMD(D, M9, Delta); /* Eq. (Hessian:F) */
        double da[3];
        if (solve3(Delta, s.f, da)) return ORC_E_LAMINATE;
        double a1[3] = {a[0] - da[0], a[1] - da[1], a[2] - da[2]}; /* naive NR update */
        double b1 = a1[0] * m[0] + a1[1] * m[1] + a1[2] * m[2];
        if (!(b1 > bcp && b1 < bcm)) {
            /* Algorithm 2: selective back-projection */
            double b0 = a[0] * m[0] + a[1] * m[1] + a[2] * m[2];
            double bc = (b1 <= bcp) ? bcp : bcm;
            double bstar = 0.5 * (b0 + bc);
            for (int i = 0; i < 3; i++) a1[i] = (a1[i] - b1 * m[i]) + bstar * m[i]; /* M_perp a1 + beta* m */
            nbp++;
        }
        a[0] = a1[0];
        a[1] = a1[1];
        a[2] = a1[2];
        it++;
        rc = lam_eval(Fb, N, cp, cm, mat, a, tol_rel, tol_abs, &s);
        if (rc) return rc;
        if (trace) {
            trace[4 * it + 0] = a[0] * m[0] + a[1] * m[1] + a[2] * m[2];
            trace[4 * it + 1] = det3(s.Fp);
            trace[4 * it + 2] = det3(s.Fm);
            trace[4 * it + 3] = s.err;
        }
    }
    for (int q = 0; q < 9; q++) P[q] = cp * s.Pp[q] + cm * s.Pm[q]; /* Eq. (Peff:Seff) */
    if (A) {
        for (int q = 0; q < 81; q++) M9[q] = s.Ap[q] / cp + s.Am[q] / cm;
        DtMD(D, M9, Delta);
        double Dinv[9];
        double dJ = det3(Delta);
        if (dJ == 0.0) return ORC_E_LAMINATE;
        inv3(Delta, dJ, Dinv);
        double dA[81], B[27], C[27], E[81];
        for (int q = 0; q < 81; q++) dA[q] = s.Ap[q] - s.Am[q];
        /* B = dA D (9x3) */
        for (int r = 0; r < 9; r++)
            for (int k = 0; k < 3; k++) {
                double t = 0.0;
                for (int q = 0; q < 9; q++) t += dA[r * 9 + q] * D[q * 3 + k];
                B[r * 3 + k] = t;
            }
        /* C = B Delta^{-1} (9x3) */
        for (int r = 0; r < 9; r++)
            for (int k = 0; k < 3; k++) {
                double t = 0.0;
                for (int q = 0; q < 3; q++) t += B[r * 3 + q] * Dinv[q * 3 + k];
                C[r * 3 + k] = t;
            }
        /* E = C D^T dA (9x9) */
        for (int r = 0; r < 9; r++)
            for (int q = 0; q < 9; q++) {
                double t = 0.0;
                for (int k = 0; k < 3; k++) {
                    double dtda = 0.0; /* (D^T dA)_{k,q} */
                    for (int w = 0; w < 9; w++) dtda += D[w * 3 + k] * dA[w * 9 + q];
                    t += C[r * 3 + k] * dtda;
                }
                E[r * 9 + q] = t;
            }
        for (int q = 0; q < 81; q++) A[q] = cp * s.Ap[q] + cm * s.Am[q] - E[q];
    }
    a_io[0] = a[0];
    a_io[1] = a[1];
    a_io[2] = a[2];
    if (iters_out) *iters_out = it;
    if (nbp_out) *nbp_out = nbp;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Infinitesimal-strain theory (cheat sheet, right column).             */
/* The stored field F is I + H (H the displacement gradient);            */
/* eps = sym(H), sigma = lam tr(eps) I + 2 mu eps = C : eps with         */
/*   C_iJkL = lam d_iJ d_kL + mu (d_ik d_JL + d_iL d_Jk).                */
/* ------------------------------------------------------------------ */
static void iso_C(double mu, double lam, double C[81])
{
    for (int i = 0; i < 3; i++)
        for (int J = 0; J < 3; J++)
            for (int k = 0; k < 3; k++)
                for (int L = 0; L < 3; L++)
                    C[9 * (3 * i + J) + 3 * k + L] =
                        lam * (i == J) * (k == L) + mu * ((i == k) * (J == L) + (i == L) * (J == k));
}

static void strain_of(const double F[9], double eps[9])
{
    for (int i = 0; i < 3; i++)
        for (int J = 0; J < 3; J++) {
            const double Hij = F[3 * i + J] - (i == J), Hji = F[3 * J + i] - (i == J);
            eps[3 * i + J] = 0.5 * (Hij + Hji);
        }
}

static void apply_C(const double C[81], const double e[9], double s[9])
{
    for (int r = 0; r < 9; r++) {
        double t = 0.0;
        for (int q = 0; q < 9; q++) t += C[9 * r + q] * e[q];
        s[r] = t;
    }
}

int orc_linear(const double F[9], double mu, double lam, double S[9], double Cout[81])
{
    double C[81], eps[9];
    iso_C(mu, lam, C);
    strain_of(F, eps);
    apply_C(C, eps, S);
    if (Cout) memcpy(Cout, C, sizeof(C));
    return ORC_OK;
}

/*
 * Infinitesimal-strain composite boxel in closed form (cheat sheet, right
 * column): Delta = N . (C+/c+ + C-/c-) . N, i.e. Delta_ik = N_J (C+/c+ + C-/c-)_iJkL N_L;
 * a = Delta^{-1} N . (C- - C+) : eps_box, i.e. a = Delta^{-1} f with f_i = ((C- - C+) : eps_box)_iJ N_J;
 * eps+- = eps_box +- sym(a (x) N) / c+-;  sigma_box = c+ sigma+ + c- sigma-;
 * C_box = (c+ C+ + c- C-) - dC (N (x) Delta^{-1} (x) N) dC, dC = C+ - C-.
 * mat = {mu-, lam-, mu+, lam+}; a receives the jump vector.
 */
int orc_laminate_linear(const double Fb[9], const double N[3], double c, const double mat[4], double a[3],
                        double S[9], double Cb[81])
{
    const double cp = c, cm = 1.0 - c;
    if (!(cp > 0.0 && cm > 0.0)) return ORC_E_INVALID;
    double Cp[81], Cm[81], eps[9];
    iso_C(mat[2], mat[3], Cp);
    iso_C(mat[0], mat[1], Cm);
    strain_of(Fb, eps);
    double Delta[9], f[3];
    for (int i = 0; i < 3; i++) {
        for (int k = 0; k < 3; k++) {
            double t = 0.0;
            for (int J = 0; J < 3; J++)
                for (int L = 0; L < 3; L++) {
                    const int r = 9 * (3 * i + J) + 3 * k + L;
                    t += N[J] * (Cp[r] / cp + Cm[r] / cm) * N[L];
                }
            Delta[3 * i + k] = t;
        }
        double t = 0.0;
        for (int J = 0; J < 3; J++)
            for (int q = 0; q < 9; q++) t += (Cm[9 * (3 * i + J) + q] - Cp[9 * (3 * i + J) + q]) * eps[q] * N[J];
        f[i] = t;
    }
    if (solve3(Delta, f, a)) return ORC_E_LAMINATE;
    double ep[9], em[9], sp[9], sm[9];
    for (int i = 0; i < 3; i++)
        for (int J = 0; J < 3; J++) {
            const double s_aN = 0.5 * (a[i] * N[J] + a[J] * N[i]);
            ep[3 * i + J] = eps[3 * i + J] + s_aN / cp;
            em[3 * i + J] = eps[3 * i + J] - s_aN / cm;
        }
    apply_C(Cp, ep, sp);
    apply_C(Cm, em, sm);
    for (int q = 0; q < 9; q++) S[q] = cp * sp[q] + cm * sm[q];
    if (Cb) {
        double Dinv[9];
        const double dJ = det3(Delta);
        if (dJ == 0.0) return ORC_E_LAMINATE;
        inv3(Delta, dJ, Dinv);
        /* B_(iJ),m = dC_iJmQ N_Q */
        double B[27];
        for (int r = 0; r < 9; r++)
            for (int m = 0; m < 3; m++) {
                double t = 0.0;
                for (int Q = 0; Q < 3; Q++) t += (Cp[9 * r + 3 * m + Q] - Cm[9 * r + 3 * m + Q]) * N[Q];
                B[3 * r + m] = t;
            }
        for (int r = 0; r < 9; r++)
            for (int q = 0; q < 9; q++) {
                double corr = 0.0;
                for (int m = 0; m < 3; m++)
                    for (int n = 0; n < 3; n++) corr += B[3 * r + m] * Dinv[3 * m + n] * B[3 * q + n];
                Cb[9 * r + q] = cp * Cp[9 * r + q] + cm * Cm[9 * r + q] - corr;
            }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* FFT: recursive mixed-radix decimation in time, full complex.         */
/* out[k] = sum_j in[j*stride] exp(sign 2 pi i j k / n).                 */
/* The twiddle table w holds exp(sign 2 pi i t / n_top) for the top-level */
/* length; a sub-transform of length n uses every (n_top/n)-th entry.     */
/* (Cooley-Tukey; the paper only uses the O(n log n) cost, Sec. 3.)        */
/* ------------------------------------------------------------------ */
static int smallest_factor(int n)
{
    for (int p = 2; p * p <= n; p++)
        if (n % p == 0) return p;
    return n;
}

static void fft_rec(const cplx* in, size_t stride, int n, const cplx* w, int wstep, cplx* out)
{
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int p = smallest_factor(n), m = n / p;
    cplx sub[n];
    for (int r = 0; r < p; r++) fft_rec(in + (size_t)r * stride, stride * p, m, w, wstep * p, sub + (size_t)r * m);
    for (int k = 0; k < n; k++) {
        cplx acc = 0.0;
        for (int r = 0; r < p; r++) acc += sub[(size_t)r * m + (k % m)] * w[(size_t)(((long)r * k) % n) * wstep];
        out[k] = acc;
    }
}

static cplx* twiddles(int n, int sign)
{
    cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    for (int t = 0; t < n; t++) {
        double ang = 2.0 * M_PI * (double)t / (double)n;
        w[t] = cos(ang) + (double)sign * I * sin(ang);
    }
    return w;
}

/* 1D transform of n points (test entry point). */
void orc_fft1(int n, int sign, const double* in_ri, double* out_ri)
{
    cplx* w = twiddles(n, sign);
    cplx* in = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    cplx* out = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    for (int j = 0; j < n; j++) in[j] = in_ri[2 * j] + I * in_ri[2 * j + 1];
    fft_rec(in, 1, n, w, 1, out);
    for (int j = 0; j < n; j++) {
        out_ri[2 * j] = creal(out[j]);
        out_ri[2 * j + 1] = cimag(out[j]);
    }
    free(w);
    free(in);
    free(out);
}

/* In-place 3D transform (no normalisation) of a complex array [n3][n2][n1]. */
static void fft3(cplx* a, const int n[3], int sign)
{
    size_t n1 = (size_t)n[0], n2 = (size_t)n[1], n3 = (size_t)n[2];
    for (int ax = 0; ax < 3; ax++) {
        size_t len = (size_t)n[ax];
        size_t stride = ax == 0 ? 1 : (ax == 1 ? n1 : n1 * n2);
        size_t nlines = n1 * n2 * n3 / len;
        cplx* w = twiddles((int)len, sign);
#pragma omp parallel for schedule(static)
        for (long li = 0; li < (long)nlines; li++) {
            size_t base;
            if (ax == 0)
                base = (size_t)li * n1;
            else if (ax == 1)
                base = ((size_t)li / n1) * n1 * n2 + ((size_t)li % n1);
            else
                base = (size_t)li;
            cplx line[len], out[len];
            for (size_t j = 0; j < len; j++) line[j] = a[base + j * stride];
            fft_rec(line, 1, (int)len, w, 1, out);
            for (size_t j = 0; j < len; j++) a[base + j * stride] = out[j];
        }
        free(w);
    }
}

void orc_fft3(const int n[3], int sign, double* data_ri)
{
    fft3((cplx*)data_ri, n, sign);
}

/* ------------------------------------------------------------------ */
/* Discrete derivative symbol k(xi) and the Green operator.             */
/* ------------------------------------------------------------------ */
#define ORC_ROTATED 0
#define ORC_SPECTRAL 1
#define ORC_STAGGERED 2
#define ORC_STAGGERED_DFMG 3 /* staggered grid with the doubly-fine material grid */

/*
 * ROTATED (Willot's rotated / HEX8R scheme, Sec. 3 and Sec. 6.3): the
 * gradient at a voxel centre is the mean of the four finite differences
 * along the edges parallel to axis j of the voxel whose corners carry the
 * displacement.  Its Fourier symbol for theta_j = 2 pi xi_j / n_j is
 *   k_j = (2 i / h_j) sin(theta_j/2) prod_{m != j} cos(theta_m/2) e^{i sum_m theta_m/2}.
 * READING: cos(theta_m/2) is set to exactly 0 at the Nyquist index xi_m = n_m/2.
 *
 * SPECTRAL (Moulinec-Suquet trigonometric polynomials, Sec. 3):
 *   k_j = 2 pi i xit_j / l_j,  xit the signed frequency;
 * READING: k_j = 0 at the Nyquist index of an even n_j.
 *
 * STAGGERED (App. A, Eqs. forward_backward_difference, gradient_operator):
 * F_aB = D_B^+ U_a on the diagonal (B = a) and D_B^- U_a off it, with
 * D^+ phi[I] = (phi[I + e_B] - phi[I]) / h_B and D^- phi[I] = (phi[I] -
 * phi[I - e_B]) / h_B; their Fourier symbols (x[I + e] <-> e^{i theta} x-hat
 * under the inverse transform's + sign) are (e^{i theta} - 1) / h and
 * (1 - e^{-i theta}) / h.  Each row a of F has its own vector k_a (the
 * diagonal entry forward, the others backward).  The rotated and spectral
 * schemes use the same k for every row.
 */
void orc_kvec(int kspace, const int n[3], const double l[3], const int xi[3], double* k_ri)
{
    cplx k[3];
    if (kspace == ORC_ROTATED) {
        double s[3], c[3], th = 0.0;
        for (int j = 0; j < 3; j++) {
            double t = 2.0 * M_PI * (double)xi[j] / (double)n[j];
            th += 0.5 * t;
            s[j] = sin(0.5 * t);
            c[j] = (2 * xi[j] == n[j]) ? 0.0 : cos(0.5 * t);
        }
        cplx ph = cos(th) + I * sin(th);
        for (int j = 0; j < 3; j++) {
            double h = l[j] / (double)n[j];
            double prod = 1.0;
            for (int m = 0; m < 3; m++)
                if (m != j) prod *= c[m];
            k[j] = (2.0 * I / h) * s[j] * prod * ph;
        }
    } else {
        for (int j = 0; j < 3; j++) {
            int x = xi[j];
            if (2 * x == n[j]) {
                k[j] = 0.0;
                continue;
            }
            int xs = (2 * x > n[j]) ? x - n[j] : x;
            k[j] = 2.0 * M_PI * I * (double)xs / l[j];
        }
    }
    for (int j = 0; j < 3; j++) {
        k_ri[2 * j] = creal(k[j]);
        k_ri[2 * j + 1] = cimag(k[j]);
    }
}

/* the derivative vector of row a of F: k_a[B], B = 0..2 */
static void row_kvecs(int kspace, const int n[3], const double l[3], const int xi[3], cplx kr[3][3])
{
    if (kspace == ORC_STAGGERED || kspace == ORC_STAGGERED_DFMG) {
        for (int B = 0; B < 3; B++) {
            const double t = 2.0 * M_PI * (double)xi[B] / (double)n[B];
            const double h = l[B] / (double)n[B];
            const cplx fwd = ((cos(t) + I * sin(t)) - 1.0) / h;
            const cplx bwd = (1.0 - (cos(t) - I * sin(t))) / h;
            for (int a = 0; a < 3; a++) kr[a][B] = (a == B) ? fwd : bwd;
        }
        return;
    }
    double k6[6];
    orc_kvec(kspace, n, l, xi, k6);
    for (int a = 0; a < 3; a++)
        for (int B = 0; B < 3; B++) kr[a][B] = k6[2 * B] + I * k6[2 * B + 1];
}

/* the derivative vector of row a (test entry point), 3 complex values */
void orc_kvec_row(int kspace, const int n[3], const double l[3], const int xi[3], int a, double* k_ri)
{
    cplx kr[3][3];
    row_kvecs(kspace, n, l, xi, kr);
    for (int B = 0; B < 3; B++) {
        k_ri[2 * B] = creal(kr[a][B]);
        k_ri[2 * B + 1] = cimag(kr[a][B]);
    }
}

/*
 * Gamma-hat for the reference medium C0 = mu0 * I4 (I4_iJkL = d_ik d_JL):
 *   Gamma0_hat_(iJ),(kL) = d_ik k_iJ conj(k_iL) / (mu0 |k_i|^2),  Gamma0_hat = 0 where k_i = 0
 * (Eq. (Gamma0): Grad G0 Div, with Div the adjoint of Grad; k_i the
 * derivative vector of row i, the same for all rows except on the staggered
 * grid).  The oracle works with G = mu0 Gamma0, the orthogonal projection
 * onto compatible zero-mean fields.  READING: C0 = mu0 I4 (the paper does not
 * fix C0); on the staggered grid Div is the adjoint of the printed Grad,
 * Div P_a = sum_B D_B^{-+} P_aB (the printed Div lists P_Ba).
 * Builds the explicit 9x9 complex matrix at one frequency; returns 0 if k=0.
 */
static int gamma_matrix(int kspace, const int n[3], const double l[3], const int xi[3], cplx Gm[81])
{
    cplx k[3][3];
    row_kvecs(kspace, n, l, xi, k);
    int any = 0;
    for (int q = 0; q < 81; q++) Gm[q] = 0.0;
    for (int i = 0; i < 3; i++) {
        double k2 = creal(k[i][0] * conj(k[i][0]) + k[i][1] * conj(k[i][1]) + k[i][2] * conj(k[i][2]));
        if (k2 == 0.0) continue;
        any = 1;
        for (int Jx = 0; Jx < 3; Jx++)
            for (int L = 0; L < 3; L++) Gm[(3 * i + Jx) * 9 + 3 * i + L] = k[i][Jx] * conj(k[i][L]) / k2;
    }
    return any;
}

/* Y = G[X] for a real 9-component field (forward FFT, 9x9 complex matrix per
 * frequency, inverse FFT / V).  Returns sum_x |Y(x)|^2 (Frobenius, summed). */
static double apply_G(int kspace, const int n[3], const double l[3], const double* X, double* Y)
{
    size_t V = (size_t)n[0] * n[1] * n[2];
    cplx* Xh = (cplx*)malloc(sizeof(cplx) * 9 * V);
    for (int c = 0; c < 9; c++) {
        for (size_t v = 0; v < V; v++) Xh[c * V + v] = X[c * V + v];
        fft3(Xh + c * V, n, -1);
    }
#pragma omp parallel for schedule(static)
    for (long v = 0; v < (long)V; v++) {
        int xi[3] = {(int)(v % n[0]), (int)((v / n[0]) % n[1]), (int)(v / ((size_t)n[0] * n[1]))};
        cplx Gm[81], in[9], out[9];
        gamma_matrix(kspace, n, l, xi, Gm);
        for (int c = 0; c < 9; c++) in[c] = Xh[c * V + v];
        for (int r = 0; r < 9; r++) {
            cplx s = 0.0;
            for (int c = 0; c < 9; c++) s += Gm[r * 9 + c] * in[c];
            out[r] = s;
        }
        for (int c = 0; c < 9; c++) Xh[c * V + v] = out[c];
    }
    double ss = 0.0;
    for (int c = 0; c < 9; c++) {
        fft3(Xh + c * V, n, +1);
        for (size_t v = 0; v < V; v++) {
            double y = creal(Xh[c * V + v]) / (double)V;
            Y[c * V + v] = y;
            ss += y * y;
        }
    }
    free(Xh);
    return ss;
}

double orc_apply_G(int kspace, const int n[3], const double l[3], const double* X, double* Y)
{
    return apply_G(kspace, n, l, X, Y);
}

/* Explicit Gamma matrix at one frequency (test entry point), 81 complex values. */
int orc_gamma_matrix(int kspace, const int n[3], const double l[3], const int xi[3], double* Gm_ri)
{
    cplx Gm[81];
    int r = gamma_matrix(kspace, n, l, xi, Gm);
    for (int q = 0; q < 81; q++) {
        Gm_ri[2 * q] = creal(Gm[q]);
        Gm_ri[2 * q + 1] = cimag(Gm[q]);
    }
    return r;
}

/* ------------------------------------------------------------------ */
/* Problem, options, result                                             */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t n[3];
    double l[3];
    const uint8_t* phase; /* [V]: 0 matrix (-), 1 inclusion (+), 2 composite boxel */
    int64_t nb;
    const int64_t* bidx; /* [nb] voxel index of each boxel */
    const double* bN;    /* [nb][3] unit normal, + -> - */
    const double* bc;    /* [nb] inclusion volume fraction c+ */
    double mu[2], lam[2];
    double Fbar[9];
    int32_t nsteps;
} orc_problem;

typedef struct {
    int32_t solver; /* 0 fixed point (basic scheme), 1 Newton-CG, 2 nonlinear CG */
    int32_t kspace; /* 0 rotated, 1 spectral, 2 staggered, 3 staggered + doubly-fine material grid */
    double tol;
    int32_t max_iter;
    int32_t fixed_iter; /* > 0: exactly this many outer iterations per load step */
    double cg_tol;
    int32_t cg_max_iter;
    int32_t cg_fixed_iter; /* > 0: exactly this many CG iterations per Newton step */
    double nr_tol_rel, nr_tol_abs;
    int32_t nr_max_iter;
    double c_min;
    double mu0; /* <= 0: default reading */
    int32_t nthreads; /* <= 0: OpenMP default */
    int32_t theory;   /* 0 finite strain (Neo-Hookean phases), 1 infinitesimal strain (isotropic linear phases) */
} orc_options;

typedef struct {
    double* Pbar;      /* [nsteps][9] */
    double* F;         /* [9][V] final step, or NULL */
    double* P;         /* [9][V] final step, or NULL */
    double* a;         /* [nb][3] final jumps, or NULL */
    int32_t* iters;    /* [nsteps] outer iterations */
    int32_t* cg_iters; /* [nsteps] CG iterations (Newton-CG) */
    double* resid;     /* [nsteps] final equilibrium residual */
    int64_t nr_iters;  /* total laminate NR iterations */
    int64_t n_backproj;
    int64_t n_lam_evals;
    int64_t n_operator; /* total operator applications (voxel-iterations / V) */
} orc_result;

/* Effective material of one voxel: laminate boxels with c outside
 * [c_min, 1 - c_min] are evaluated as the pure phase they almost are
 * (READING; the paper's 5..95 % cut-off is what it argues against, so
 * c_min is tiny). */
typedef struct {
    const orc_problem* pb;
    const orc_options* op;
    int32_t* vox2box; /* [V] boxel index or -1 */
    double* a;        /* [nb][3] jump vectors (warm start state) */
    double* a8;       /* doubly-fine material grid: [nb][8][3] jump vectors of the sub-cells */
} orc_ctx;

/* Material law of cell v at Fs (pure Neo-Hookean, or the laminate of a boxel
 * cell from the warm start a_ws, updated). */
static int cell_law(orc_ctx* cx, long v, const double Fs[9], double a_ws[3], double P[9], double* A,
                    int64_t* its_o, int64_t* nbp_o)
{
    const orc_problem* pb = cx->pb;
    int b = cx->vox2box[v];
    int ph = pb->phase[v];
    double cpl = 0.0;
    if (b >= 0) {
        cpl = pb->bc[b];
        if (cpl < cx->op->c_min) ph = 0;
        else if (cpl > 1.0 - cx->op->c_min) ph = 1;
    }
    if (ph == 2) {
        double mat[4] = {pb->mu[0], pb->lam[0], pb->mu[1], pb->lam[1]};
        int its = 0, nbpv = 0;
        int rc = orc_laminate(Fs, pb->bN + 3 * (size_t)b, cpl, mat, a_ws, cx->op->nr_tol_rel, cx->op->nr_tol_abs,
                              cx->op->nr_max_iter, P, A, &its, &nbpv, NULL);
        *its_o += its;
        *nbp_o += nbpv;
        return rc;
    }
    return orc_neohooke(Fs, pb->mu[ph], pb->lam[ph], P, A);
}

static long wrapi(long i, long n) { return ((i % n) + n) % n; }

/* F_sub(c, l) of the field X [9][V] at cell v (see constitutive_dfmg). */
static void dfmg_assemble(const orc_problem* pb, const double* X, long v, int l, double out[9])
{
    const long n1 = pb->n[0], n2 = pb->n[1], n3 = pb->n[2];
    const size_t V = (size_t)n1 * n2 * n3;
    const long i = v % n1, j = (v / n1) % n2, k = v / (n1 * n2);
    const long l1 = l & 1, l2 = (l >> 1) & 1, l3 = (l >> 2) & 1;
    const long v12 = wrapi(i + l1, n1) + n1 * (wrapi(j + l2, n2) + n2 * k);
    const long v13 = wrapi(i + l1, n1) + n1 * (j + n2 * wrapi(k + l3, n3));
    const long v23 = i + n1 * (wrapi(j + l2, n2) + n2 * wrapi(k + l3, n3));
    out[0] = X[0 * V + v];
    out[4] = X[4 * V + v];
    out[8] = X[8 * V + v];
    out[1] = X[1 * V + v12];
    out[3] = X[3 * V + v12];
    out[2] = X[2 * V + v13];
    out[6] = X[6 * V + v13];
    out[5] = X[5 * V + v23];
    out[7] = X[7 * V + v23];
}

/* The gather of the sub-cell values S [V][8][9] into Y [9][V] (see
 * constitutive_dfmg): diagonal from the cell's own sub-cells, off-diagonal
 * (a, b) of sub-cell l from the cell xi - l_a e_a - l_b e_b. */
static void dfmg_gather(const orc_problem* pb, const double* S, double* Y)
{
    const long n1 = pb->n[0], n2 = pb->n[1], n3 = pb->n[2];
    const size_t V = (size_t)n1 * n2 * n3;
#pragma omp parallel for schedule(static)
    for (long v = 0; v < (long)V; v++) {
        const long i = v % n1, j = (v / n1) % n2, k = v / (n1 * n2);
        double out[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int l = 0; l < 8; l++) {
            const long l1 = l & 1, l2 = (l >> 1) & 1, l3 = (l >> 2) & 1;
            const double* Sv = S + 72 * (size_t)v + 9 * l;
            out[0] += Sv[0];
            out[4] += Sv[4];
            out[8] += Sv[8];
            const long c12 = wrapi(i - l1, n1) + n1 * (wrapi(j - l2, n2) + n2 * k);
            const long c13 = wrapi(i - l1, n1) + n1 * (j + n2 * wrapi(k - l3, n3));
            const long c23 = i + n1 * (wrapi(j - l2, n2) + n2 * wrapi(k - l3, n3));
            out[1] += S[72 * (size_t)c12 + 9 * l + 1];
            out[3] += S[72 * (size_t)c12 + 9 * l + 3];
            out[2] += S[72 * (size_t)c13 + 9 * l + 2];
            out[6] += S[72 * (size_t)c13 + 9 * l + 6];
            out[5] += S[72 * (size_t)c23 + 9 * l + 5];
            out[7] += S[72 * (size_t)c23 + 9 * l + 7];
        }
        for (int c = 0; c < 9; c++) Y[(size_t)c * V + v] = 0.125 * out[c];
    }
}

/*
 * Doubly-fine material grid (App. A, Eq. constitutive_law): every cell is cut
 * into 8 sub-cells l = (l1, l2, l3) in {0,1}^3; sub-cell l of cell c carries the
 * deformation gradient F_sub(c, l) whose diagonal entries are those of the
 * cell centre c and whose off-diagonal entries come from the nearest staggered
 * positions: F_12, F_21 from c + (l1, l2, 0), F_13, F_31 from c + (l1, 0, l3),
 * F_23, F_32 from c + (0, l2, l3) (the F^{aa}_l of the paper).  The law is
 *   P_aa[xi] = 1/8 sum_l P_xi(F_sub(xi, l))_aa,
 *   P_ab[xi] = 1/8 sum_l P_c(F_sub(c, l))_ab, c = xi - l_a e_a - l_b e_b (a != b),
 * which is the paper's F^{ab}_l[xi] assembly (F_sub(c, l) with that c) with the
 * material of the cell that holds the sub-cell.  READING: the paper prints the
 * material P[xi + l^{+a,+b}], whose offsets disagree in sign with those of
 * F^{ab}_l; with xi - l_a e_a - l_b e_b the law is the gradient of the sub-cell
 * energy 1/8 sum_c sum_l W_c(F_sub(c, l)) (pinned by finite differences).
 * Each sub-cell's law is evaluated once (S below) and gathered per the
 * equation; boxel cells keep one jump-vector warm start per sub-cell.
 */
static int constitutive_dfmg(orc_ctx* cx, const double* F, double* P, double* A8, int64_t* nr_it, int64_t* nbp,
                             int64_t* nevals)
{
    const orc_problem* pb = cx->pb;
    size_t V = (size_t)pb->n[0] * pb->n[1] * pb->n[2];
    double* S = (double*)malloc(sizeof(double) * 72 * V); /* [V][8][9] */
    int status = ORC_OK;
    int64_t it_sum = 0, bp_sum = 0, ev_sum = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : it_sum, bp_sum, ev_sum)
    for (long v = 0; v < (long)V; v++) {
        const int b = cx->vox2box[v];
        for (int l = 0; l < 8; l++) {
            double Fs[9];
            dfmg_assemble(pb, F, v, l, Fs);
            double aw[3] = {0.0, 0.0, 0.0};
            if (b >= 0) memcpy(aw, cx->a8 + 24 * (size_t)b + 3 * l, sizeof(aw));
            int64_t its = 0, nbpv = 0;
            int rc = cell_law(cx, v, Fs, aw, S + 72 * (size_t)v + 9 * l, A8 ? A8 + 81 * (8 * (size_t)v + l) : NULL,
                              &its, &nbpv);
            if (b >= 0) {
                memcpy(cx->a8 + 24 * (size_t)b + 3 * l, aw, sizeof(aw));
                ev_sum += 1;
            }
            it_sum += its;
            bp_sum += nbpv;
            if (rc) {
#pragma omp critical
                {
                    if (status == ORC_OK) status = rc;
                }
            }
        }
    }
    if (status == ORC_OK) dfmg_gather(pb, S, P);
    free(S);
    if (nr_it) *nr_it += it_sum;
    if (nbp) *nbp += bp_sum;
    if (nevals) *nevals += ev_sum;
    return status;
}

/* Tangent of the doubly-fine law applied to a field X [9][V]: with the
 * sub-cell tangents A8 [V][8][81] of the last law evaluation, Y = the gather
 * of A_sub(c, l) : X_sub(c, l), X_sub assembled like F_sub.  It is the
 * Hessian of the sub-cell energy, hence symmetric (pinned). */
static void dfmg_tangent_apply(const orc_problem* pb, const double* A8, const double* X, double* Y)
{
    size_t V = (size_t)pb->n[0] * pb->n[1] * pb->n[2];
    double* S = (double*)malloc(sizeof(double) * 72 * V);
#pragma omp parallel for schedule(static)
    for (long v = 0; v < (long)V; v++) {
        for (int l = 0; l < 8; l++) {
            double xs[9];
            dfmg_assemble(pb, X, v, l, xs);
            const double* Al = A8 + 81 * (8 * (size_t)v + l);
            for (int r = 0; r < 9; r++) {
                double t = 0.0;
                for (int c = 0; c < 9; c++) t += Al[9 * r + c] * xs[c];
                S[72 * (size_t)v + 9 * l + r] = t;
            }
        }
    }
    dfmg_gather(pb, S, Y);
    free(S);
}
/* Reported jump vector of a boxel under the doubly-fine material grid: the
 * mean of its 8 sub-cell jumps (the sub-cell jumps themselves are internal
 * warm-start state). */
static void dfmg_mean_jumps(const double* a8, int64_t nb, double* a)
{
    for (int64_t b = 0; b < nb; b++)
        for (int q = 0; q < 3; q++) {
            double s = 0.0;
            for (int l = 0; l < 8; l++) s += a8[24 * b + 3 * l + q];
            a[3 * b + q] = 0.125 * s;
        }
}

/* P (and optionally the 9x9 tangent A) at every voxel.  Returns status. */
static int constitutive(orc_ctx* cx, const double* F, double* P, double* A, int64_t* nr_it, int64_t* nbp,
                        int64_t* nevals)
{
    const orc_problem* pb = cx->pb;
    if (cx->op->kspace == ORC_STAGGERED_DFMG) /* A, if given, receives the sub-cell tangents [V][8][81] */
        return constitutive_dfmg(cx, F, P, A, nr_it, nbp, nevals);
    size_t V = (size_t)pb->n[0] * pb->n[1] * pb->n[2];
    int status = ORC_OK;
    int64_t it_sum = 0, bp_sum = 0, ev_sum = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : it_sum, bp_sum, ev_sum)
    for (long v = 0; v < (long)V; v++) {
        double Fv[9], Pv[9], Av[81];
        for (int c = 0; c < 9; c++) Fv[c] = F[(size_t)c * V + v];
        int rc;
        int b = cx->vox2box[v];
        int ph = pb->phase[v];
        double cpl = 0.0;
        if (b >= 0) {
            cpl = pb->bc[b];
            if (cpl < cx->op->c_min) ph = 0;
            else if (cpl > 1.0 - cx->op->c_min) ph = 1;
        }
        if (cx->op->theory == 1) {
            if (ph == 2) {
                double mat[4] = {pb->mu[0], pb->lam[0], pb->mu[1], pb->lam[1]};
                rc = orc_laminate_linear(Fv, pb->bN + 3 * (size_t)b, cpl, mat, cx->a + 3 * (size_t)b, Pv,
                                         A ? Av : NULL);
                ev_sum += 1;
            } else {
                rc = orc_linear(Fv, pb->mu[ph], pb->lam[ph], Pv, A ? Av : NULL);
            }
        } else if (ph == 2) {
            double mat[4] = {pb->mu[0], pb->lam[0], pb->mu[1], pb->lam[1]};
            int its = 0, nbpv = 0;
            rc = orc_laminate(Fv, pb->bN + 3 * (size_t)b, cpl, mat, cx->a + 3 * (size_t)b, cx->op->nr_tol_rel,
                              cx->op->nr_tol_abs, cx->op->nr_max_iter, Pv, A ? Av : NULL, &its, &nbpv, NULL);
            it_sum += its;
            bp_sum += nbpv;
            ev_sum += 1;
        } else {
            rc = orc_neohooke(Fv, pb->mu[ph], pb->lam[ph], Pv, A ? Av : NULL);
        }
        if (rc) {
#pragma omp critical
            {
                if (status == ORC_OK) status = rc;
            }
            continue;
        }
        for (int c = 0; c < 9; c++) P[(size_t)c * V + v] = Pv[c];
        if (A) memcpy(A + (size_t)v * 81, Av, sizeof(double) * 81);
    }
    if (nr_it) *nr_it += it_sum;
    if (nbp) *nbp += bp_sum;
    if (nevals) *nevals += ev_sum;
    return status;
}

int orc_constitutive_field(const orc_problem* pb, const orc_options* op, const double* F, double* a_io, double* P,
                           double* A)
{
    if (A && op->kspace == ORC_STAGGERED_DFMG) return ORC_E_INVALID; /* no per-voxel tangent: orc_dfmg_tangent_apply */
    size_t V = (size_t)pb->n[0] * pb->n[1] * pb->n[2];
    orc_ctx cx = {pb, op, (int32_t*)malloc(sizeof(int32_t) * V), a_io,
                  (double*)calloc(24 * (size_t)(pb->nb > 0 ? pb->nb : 1), sizeof(double))};
    for (size_t v = 0; v < V; v++) cx.vox2box[v] = -1;
    for (int64_t b = 0; b < pb->nb; b++) cx.vox2box[pb->bidx[b]] = (int32_t)b;
    int rc = constitutive(&cx, F, P, A, NULL, NULL, NULL);
    if (op->kspace == ORC_STAGGERED_DFMG) dfmg_mean_jumps(cx.a8, pb->nb, a_io);
    free(cx.vox2box);
    free(cx.a8);
    return rc;
}

/* The tangent of the doubly-fine law at F applied to X: Y = dP/dF [X]
 * (test entry of dfmg_tangent_apply; boxel sub-cells start from a = 0). */
int orc_dfmg_tangent_apply(const orc_problem* pb, const orc_options* op, const double* F, const double* X, double* Y)
{
    size_t V = (size_t)pb->n[0] * pb->n[1] * pb->n[2];
    orc_ctx cx = {pb, op, (int32_t*)malloc(sizeof(int32_t) * V), NULL,
                  (double*)calloc(24 * (size_t)(pb->nb > 0 ? pb->nb : 1), sizeof(double))};
    for (size_t v = 0; v < V; v++) cx.vox2box[v] = -1;
    for (int64_t b = 0; b < pb->nb; b++) cx.vox2box[pb->bidx[b]] = (int32_t)b;
    double* A8 = (double*)malloc(sizeof(double) * 648 * V);
    double* P = (double*)malloc(sizeof(double) * 9 * V);
    int rc = constitutive_dfmg(&cx, F, P, A8, NULL, NULL, NULL);
    if (rc == ORC_OK) dfmg_tangent_apply(pb, A8, X, Y);
    free(P);
    free(A8);
    free(cx.vox2box);
    free(cx.a8);
    return rc;
}

static void field_mean(const double* X, size_t V, double m[9])
{
    for (int c = 0; c < 9; c++) {
        double s = 0.0;
        for (size_t v = 0; v < V; v++) s += X[(size_t)c * V + v];
        m[c] = s / (double)V;
    }
}

static double dot(const double* x, const double* y, size_t n)
{
    double s = 0.0;
    for (size_t i = 0; i < n; i++) s += x[i] * y[i];
    return s;
}

/* y = A : x at every voxel, A dense 9x9 per voxel. */
static void tangent_apply(const double* A, const double* x, double* y, size_t V)
{
#pragma omp parallel for schedule(static)
    for (long v = 0; v < (long)V; v++) {
        const double* Av = A + (size_t)v * 81;
        for (int r = 0; r < 9; r++) {
            double s = 0.0;
            for (int c = 0; c < 9; c++) s += Av[r * 9 + c] * x[(size_t)c * V + v];
            y[(size_t)r * V + v] = s;
        }
    }
}

/* All J > 0: pure voxels det F; boxels det F_box (a = 0 is then admissible). */
static int all_admissible(const double* F, size_t V)
{
    int ok = 1;
#pragma omp parallel for schedule(static) reduction(&& : ok)
    for (long v = 0; v < (long)V; v++) {
        double Fv[9];
        for (int c = 0; c < 9; c++) Fv[c] = F[(size_t)c * V + v];
        ok = ok && (det3(Fv) > 0.0);
    }
    return ok;
}

/*
 * Full solve of the homogenization problem (HOM), Sec. 2, by the
 * Lippmann-Schwinger equation of Sec. 3, Eq. (nonlinearLSE).
 *
 * Load stepping (READING; the paper is silent): Fbar_n = I + (n/S)(Fbar - I),
 * n = 1..S; the new step starts from the previous field plus the uniform
 * increment Fbar_n - Fbar_{n-1}.
 *
 * Equilibrium residual (READING): eps = ||G[P]||_rms / ||<P>||_F, where
 * ||.||_rms is the root mean square over voxels of the Frobenius norm.
 *
 * Fixed point (solver 0): the basic scheme applied to the nonlinear LSE
 * (Sec. 3): F <- F - Gamma0 (P(F)) = F - G[P(F)] / mu0 for compatible F with
 * mean Fbar.  READING: mu0 = (min mu + max(lam + 2 mu)) / 2.
 *
 * Nonlinear CG (solver 2; Sec. 3 cites it, the paper gives no steps): the
 * Fletcher-Reeves nonlinear conjugate gradient method on the energy over
 * compatible fields, with the basic scheme's preconditioned gradient
 * G[P(F)] / mu0 and its step length: d = -G[P]/mu0 + beta d_prev,
 * beta = ||G[P]||^2 / ||G[P_prev]||^2 (0 at a load step's first iteration),
 * F += d.  READING: Fletcher-Reeves, no line search.
 *
 * Newton-CG (solver 1): Newton on G[P(F)] = 0 with the linearised system
 * G[A : dF] = -G[P] solved by conjugate gradients in the Frobenius inner
 * product on compatible zero-mean fields (Sec. 3, Newton with a fast linear
 * solver).  CG stops when ||r|| <= cg_tol ||b||.  If a Newton update makes
 * any det F <= 0 the update is halved, at most 10 times.
 */
int orc_solve(const orc_problem* pb, const orc_options* op, orc_result* res)
{
#ifdef _OPENMP
    if (op->nthreads > 0) omp_set_num_threads(op->nthreads);
#endif
    const int* n = pb->n;
    size_t V = (size_t)n[0] * n[1] * n[2];
    size_t N9 = 9 * V;
    orc_ctx cx;
    cx.pb = pb;
    cx.op = op;
    cx.vox2box = (int32_t*)malloc(sizeof(int32_t) * V);
    for (size_t v = 0; v < V; v++) cx.vox2box[v] = -1;
    for (int64_t b = 0; b < pb->nb; b++) cx.vox2box[pb->bidx[b]] = (int32_t)b;
    cx.a = (double*)calloc(3 * (size_t)(pb->nb > 0 ? pb->nb : 1), sizeof(double));
    cx.a8 = (double*)calloc(24 * (size_t)(pb->nb > 0 ? pb->nb : 1), sizeof(double));
    if (op->kspace == ORC_STAGGERED_DFMG && op->theory == 1) {
        free(cx.vox2box);
        free(cx.a);
        free(cx.a8);
        return ORC_E_INVALID; /* Newton needs the tangent, which the DFMG law does not provide here */
    }

    double* F = (double*)malloc(sizeof(double) * N9);
    double* P = (double*)malloc(sizeof(double) * N9);
    double* g = (double*)malloc(sizeof(double) * N9);
    double* A = NULL;
    double *x = NULL, *r = NULL, *p = NULL, *q = NULL, *t = NULL, *dir = NULL;
    if (op->solver == 2) dir = (double*)calloc(N9, sizeof(double));
    if (op->solver == 1) {
        /* (the doubly-fine grid keeps one tangent per sub-cell) */
        A = (double*)malloc(sizeof(double) * 81 * V * (op->kspace == ORC_STAGGERED_DFMG ? 8 : 1));
        x = (double*)malloc(sizeof(double) * N9);
        r = (double*)malloc(sizeof(double) * N9);
        p = (double*)malloc(sizeof(double) * N9);
        q = (double*)malloc(sizeof(double) * N9);
        t = (double*)malloc(sizeof(double) * N9);
    }
    double mu0 = op->mu0;
    if (!(mu0 > 0.0)) {
        double mumin = fmin(pb->mu[0], pb->mu[1]);
        double pmax = fmax(pb->lam[0] + 2 * pb->mu[0], pb->lam[1] + 2 * pb->mu[1]);
        mu0 = 0.5 * (mumin + pmax);
    }
    static const double Id[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int c = 0; c < 9; c++)
        for (size_t v = 0; v < V; v++) F[(size_t)c * V + v] = Id[c];
    double Fprev[9];
    memcpy(Fprev, Id, sizeof(Fprev));
    int status = ORC_OK;
    res->nr_iters = res->n_backproj = res->n_lam_evals = res->n_operator = 0;

    for (int step = 1; step <= pb->nsteps && status == ORC_OK; step++) {
        double Fn[9];
        for (int c = 0; c < 9; c++) Fn[c] = Id[c] + ((double)step / pb->nsteps) * (pb->Fbar[c] - Id[c]);
        for (int c = 0; c < 9; c++) {
            double d = Fn[c] - Fprev[c];
            for (size_t v = 0; v < V; v++) F[(size_t)c * V + v] += d;
        }
        memcpy(Fprev, Fn, sizeof(Fn));
        int it = 0, cg_total = 0;
        double eps = 0.0, Pbar[9], gg_prev = 0.0;
        for (;;) {
            int rc = constitutive(&cx, F, P, A, &res->nr_iters, &res->n_backproj, &res->n_lam_evals);
            if (rc) {
                status = rc;
                break;
            }
            field_mean(P, V, Pbar);
            double ss = apply_G(op->kspace, n, pb->l, P, g);
            double pn = sqrt(dot(Pbar, Pbar, 9));
            eps = sqrt(ss / (double)V) / (pn > 0.0 ? pn : 1.0);
            if (!isfinite(eps)) {
                status = ORC_E_NAN;
                break;
            }
            if (op->fixed_iter > 0 ? it >= op->fixed_iter : eps <= op->tol) break;
            if (it >= op->max_iter) {
                status = ORC_E_NOT_CONVERGED;
                break;
            }
            if (op->solver == 0) {
                for (size_t w = 0; w < N9; w++) F[w] -= g[w] / mu0;
                res->n_operator += 1;
            } else if (op->solver == 2) {
                const double beta = (it == 0) ? 0.0 : ss / gg_prev;
                for (size_t w = 0; w < N9; w++) {
                    dir[w] = -g[w] / mu0 + beta * dir[w];
                    F[w] += dir[w];
                }
                gg_prev = ss;
                res->n_operator += 1;
            } else {
                /* CG on G[A : x] = b, b = -G[P] */
                for (size_t w = 0; w < N9; w++) {
                    x[w] = 0.0;
                    r[w] = -g[w];
                    p[w] = r[w];
                }
                double rr = dot(r, r, N9), rr0 = rr;
                int j = 0;
                for (;;) {
                    if (op->cg_fixed_iter > 0) {
                        if (j >= op->cg_fixed_iter) break;
                    } else if (sqrt(rr) <= op->cg_tol * sqrt(rr0) || j >= op->cg_max_iter)
                        break;
                    if (rr == 0.0) break;
                    if (op->kspace == ORC_STAGGERED_DFMG)
                        dfmg_tangent_apply(pb, A, p, t);
                    else
                        tangent_apply(A, p, t, V);
                    apply_G(op->kspace, n, pb->l, t, q);
                    res->n_operator += 1;
                    double pq = dot(p, q, N9);
                    if (!(pq > 0.0)) break; /* READING: stop CG on loss of positive curvature */
                    double alpha = rr / pq;
                    for (size_t w = 0; w < N9; w++) {
                        x[w] += alpha * p[w];
                        r[w] -= alpha * q[w];
                    }
                    double rr_new = dot(r, r, N9);
                    double beta = rr_new / rr;
                    rr = rr_new;
                    for (size_t w = 0; w < N9; w++) p[w] = r[w] + beta * p[w];
                    j++;
                }
                cg_total += j;
                /* F <- F + s x with s = 1, 1/2, ... keeping det F > 0 */
                double s = 1.0;
                int ok = 0;
                for (int h = 0; h <= 10; h++) {
                    for (size_t w = 0; w < N9; w++) t[w] = F[w] + s * x[w];
                    if (op->theory == 1 || all_admissible(t, V)) { /* (no det F constraint on small strains) */
                        ok = 1;
                        break;
                    }
                    s *= 0.5;
                }
                if (!ok) {
                    status = ORC_E_INADMISSIBLE;
                    break;
                }
                memcpy(F, t, sizeof(double) * N9);
            }
            it++;
        }
        memcpy(res->Pbar + 9 * (size_t)(step - 1), Pbar, sizeof(Pbar));
        if (res->iters) res->iters[step - 1] = it;
        if (res->cg_iters) res->cg_iters[step - 1] = cg_total;
        if (res->resid) res->resid[step - 1] = eps;
    }
    if (res->F) memcpy(res->F, F, sizeof(double) * N9);
    if (res->P) memcpy(res->P, P, sizeof(double) * N9);
    if (op->kspace == ORC_STAGGERED_DFMG) dfmg_mean_jumps(cx.a8, pb->nb, cx.a);
    if (res->a && pb->nb > 0) memcpy(res->a, cx.a, sizeof(double) * 3 * (size_t)pb->nb);
    free(cx.vox2box);
    free(cx.a);
    free(cx.a8);
    free(F);
    free(P);
    free(g);
    free(A);
    free(x);
    free(r);
    free(p);
    free(q);
    free(t);
    free(dir);
    return status;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
