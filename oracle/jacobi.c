/*
 * oracle/jacobi.c -- cyclic Jacobi eigensolver for the FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file belongs to the oracle that the test
 * suite, __graft_entry__.smoke() and bench.py's CPU-baseline leg use to check
 * the CUDA path.  The product library never includes, links or calls it, and
 * it shares no code with the CUDA sources.
 *
 * What it computes: the "full-PCA" step of primed PCA (Algorithm 1, step 4,
 * Section 3.2) and the ground-truth principal directions (Section 1: the
 * principal directions are the eigenvectors of the covariance matrix X^T X)
 * both reduce to the eigendecomposition of a real symmetric matrix.  This is
 * the textbook cyclic-by-row Jacobi method: sweep over the pairs (p, q),
 * p < q, in row order; for each pair apply the plane rotation that zeroes
 * a_pq, with the classical choice of the smaller rotation angle
 *     tau = (a_qq - a_pp) / (2 a_pq),
 *     t   = sign(tau) / (|tau| + sqrt(1 + tau^2)),
 *     c   = 1 / sqrt(1 + t^2),   s = t c,
 * and accumulate the rotations into V.  Plain double precision, no blocking.
 */
#include <math.h>
#include <stddef.h>

static double off_norm2(const double *A, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (i != j)
                s += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    return s;
}

static double fro_norm2(const double *A, int n)
{
    double s = 0.0;
    for (size_t i = 0; i < (size_t)n * n; ++i)
        s += A[i] * A[i];
    return s;
}

/*
 * A: n x n symmetric, row-major; overwritten, its diagonal holds the
 *    eigenvalues on return (unsorted).
 * V: n x n row-major; on return column j is the unit eigenvector of A[j][j].
 * Stops when off(A) <= tol * ||A||_F, or when a whole sweep finds every
 * off-diagonal entry negligible (|a_pq| <= 1e-300, or |a_pq| below
 * 2^-53 * sqrt(|a_pp a_qq|) so that the rotation cannot change the diagonal).
 * Returns the number of sweeps done, or -1 if max_sweeps ran out first.
 */
int oracle_jacobi_cyclic(double *A, double *V, int n, double tol, int max_sweeps)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            V[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
    if (n <= 1)
        return 0;
    const double fro = sqrt(fro_norm2(A, n));
    const double eps = ldexp(1.0, -53);
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (sqrt(off_norm2(A, n)) <= tol * fro)
            return sweep;
        int rotated = 0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                const double app = A[(size_t)p * n + p];
                const double aqq = A[(size_t)q * n + q];
                if (fabs(apq) <= 1e-300 || fabs(apq) <= eps * sqrt(fabs(app * aqq)))
                    continue;
                rotated = 1;
                const double tau = (aqq - app) / (2.0 * apq);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t);
                const double s = t * c;
                /* columns p, q of A: A <- A J */
                for (int r = 0; r < n; ++r) {
                    const double arp = A[(size_t)r * n + p];
                    const double arq = A[(size_t)r * n + q];
                    A[(size_t)r * n + p] = c * arp - s * arq;
                    A[(size_t)r * n + q] = s * arp + c * arq;
                }
                /* rows p, q of A: A <- J^T A */
                for (int r = 0; r < n; ++r) {
                    const double apr = A[(size_t)p * n + r];
                    const double aqr = A[(size_t)q * n + r];
                    A[(size_t)p * n + r] = c * apr - s * aqr;
                    A[(size_t)q * n + r] = s * apr + c * aqr;
                }
                /* the rotation zeroes a_pq exactly in exact arithmetic */
                A[(size_t)p * n + q] = 0.0;
                A[(size_t)q * n + p] = 0.0;
                for (int r = 0; r < n; ++r) {
                    const double vrp = V[(size_t)r * n + p];
                    const double vrq = V[(size_t)r * n + q];
                    V[(size_t)r * n + p] = c * vrp - s * vrq;
                    V[(size_t)r * n + q] = s * vrp + c * vrq;
                }
            }
        }
        if (!rotated)
            return sweep + 1;
    }
    if (sqrt(off_norm2(A, n)) <= tol * fro)
        return max_sweeps;
    return -1;
}

/* Version tag so the Python side can check it loaded this file's build. */
int oracle_jacobi_abi_version(void) { return 1; }
