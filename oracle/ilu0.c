/*
 * Plain CPU ILU(0) for the oracle (test infrastructure only: only the tests, the
 * smoke check and the benchmark's CPU-baseline leg load this file's library).
 *
 * The subdomain solver of the Schwarz preconditioner (Sec. 3.1, Eq. invM and the
 * text after it) applies inv(A_k) through an incomplete LU factorisation with
 * zero fill-in.  This is the textbook IKJ form of ILU(0) on a CSR matrix whose
 * column indices are sorted in every row: the factors keep exactly the sparsity
 * pattern of A (explicit zeros included), L has a unit diagonal and is stored
 * below the diagonal, U on and above it.  Written from the definition of ILU(0):
 * Gaussian elimination in natural row order in which every update that would
 * land outside the pattern of A is dropped.
 */
#include <stdlib.h>

/* Factor in place.  diag[i] receives the position of a_ii.
 * Returns 0, -1 on allocation failure, or -(i+2) if pivot i is missing or zero. */
int oracle_ilu0_factor(int n, const int *indptr, const int *indices, double *a, int *diag)
{
    int *pos = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    if (!pos) return -1;
    for (int i = 0; i < n; i++) pos[i] = -1;
    int status = 0;
    for (int i = 0; i < n && status == 0; i++) {
        for (int p = indptr[i]; p < indptr[i + 1]; p++) pos[indices[p]] = p;
        /* eliminate the entries left of the diagonal, in increasing column order */
        for (int p = indptr[i]; p < indptr[i + 1]; p++) {
            int k = indices[p];
            if (k >= i) break;
            a[p] /= a[diag[k]];
            /* row i -= l_ik * (upper part of row k), only where row i has an entry */
            for (int q = diag[k] + 1; q < indptr[k + 1]; q++) {
                int j = indices[q];
                if (pos[j] >= 0) a[pos[j]] -= a[p] * a[q];
            }
        }
        int d = pos[i];
        if (d < 0 || a[d] == 0.0) status = -(i + 2);
        else diag[i] = d;
        for (int p = indptr[i]; p < indptr[i + 1]; p++) pos[indices[p]] = -1;
    }
    free(pos);
    return status;
}

/* Solve (LU) x = b with the factors above: forward with unit-lower L, then backward. */
void oracle_ilu0_solve(int n, const int *indptr, const int *indices, const double *a,
                       const int *diag, const double *b, double *x)
{
    for (int i = 0; i < n; i++) {
        double s = b[i];
        for (int p = indptr[i]; p < diag[i]; p++) s -= a[p] * x[indices[p]];
        x[i] = s;
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = x[i];
        for (int p = diag[i] + 1; p < indptr[i + 1]; p++) s -= a[p] * x[indices[p]];
        x[i] = s / a[diag[i]];
    }
}
