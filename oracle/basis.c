/*
 * Oracle, C part: explicit sorted basis, binary lookup and CSR Hamiltonian.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct CPU
 * restatement of the paper's construction, used by tests/, by __graft_entry__.smoke()
 * and by bench.py's CPU-baseline leg.  The product path never links or calls it, and
 * it shares no code, header or table with the CUDA library.
 *
 * What it follows:
 *   - Sec. 2 "Basis representation": a state is an integer whose bit i-1 is the
 *     occupation of site i; the sector with N particles has D = L!/(N!(L-N)!) states.
 *   - Algorithm 2 (ConstructIntBasis): sorted basis by next permutation of bits,
 *     starting at the smallest integer 2^N - 1.  The printed expression is garbled in
 *     its precedence; it is read as  t = (v | (v-1)) + 1;
 *     w = t | ((((t & -t) / (v & -v)) >> 1) - 1).
 *   - Sec. 3 "Hamiltonian matrix construction": apply the Hamiltonian to every basis
 *     state with bit operations and find column indices by binary lookup in the sorted
 *     basis.
 *   - Eq. 1 in its XXZ form: H = J sum_b [ (S+_i S-_j + h.c.)/2 + Delta Sz_i Sz_j ]
 *     + sum_i h_i Sz_i, with Sz = n - 1/2.  Bonds b = (i, i+1) for i = 0..L-2, plus the
 *     ring bond (L-1, 0) when periodic and L >= 3.
 */
#include <stdint.h>
#include <stdlib.h>

/* Binomial coefficient by the multiplicative formula (exact for the sizes used here). */
int64_t orc_binom(int n, int k)
{
    if (k < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

/* Algorithm 2: fill out[0..D-1] with the sorted basis of the (L, N) sector.
 * Returns D, or -1 if cap < D or the sizes are out of range. */
int64_t orc_basis(int L, int N, uint64_t *out, int64_t cap)
{
    if (L < 1 || L > 62 || N < 0 || N > L) return -1;
    int64_t D = orc_binom(L, N);
    if (cap < D) return -1;
    uint64_t v = (N == 0) ? 0 : ((N == 64) ? ~0ull : ((1ull << N) - 1ull)); /* smallest_int() */
    out[0] = v;
    for (int64_t i = 1; i < D; ++i) {
        uint64_t t = (v | (v - 1ull)) + 1ull;
        uint64_t w = t | ((((t & (~t + 1ull)) / (v & (~v + 1ull))) >> 1) - 1ull);
        out[i] = w;
        v = w;
    }
    return D;
}

/* Binary lookup of state s in the sorted basis; returns its index or -1. */
int64_t orc_lookup(const uint64_t *basis, int64_t D, uint64_t s)
{
    int64_t lo = 0, hi = D - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (basis[mid] == s) return mid;
        if (basis[mid] < s) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

static int n_bonds(int L, int pbc) { return (pbc && L >= 3) ? L : (L - 1 > 0 ? L - 1 : 0); }

static void bond_sites(int b, int L, int *i, int *j)
{
    *i = b;
    *j = (b + 1 < L) ? b + 1 : 0;   /* b = L-1 is the ring bond (L-1, 0) */
}

/* Number of stored entries of row `state` (diagonal always stored). */
static int64_t row_nnz(uint64_t s, int L, int pbc)
{
    int64_t c = 1;
    int nb = n_bonds(L, pbc);
    for (int b = 0; b < nb; ++b) {
        int i, j;
        bond_sites(b, L, &i, &j);
        if (((s >> i) & 1ull) != ((s >> j) & 1ull)) ++c;
    }
    return c;
}

/* Counting pass: total stored entries of the CSR matrix. */
int64_t orc_ham_nnz(int L, const uint64_t *basis, int64_t D, int pbc)
{
    int64_t nnz = 0;
    for (int64_t r = 0; r < D; ++r) nnz += row_nnz(basis[r], L, pbc);
    return nnz;
}

/* Diagonal element of Eq. 1 (XXZ form) for state s. */
double orc_diag(uint64_t s, int L, double J, double Delta, const double *h, int pbc)
{
    double d = 0.0;
    int nb = n_bonds(L, pbc);
    for (int b = 0; b < nb; ++b) {
        int i, j;
        bond_sites(b, L, &i, &j);
        double szi = ((s >> i) & 1ull) ? 0.5 : -0.5;
        double szj = ((s >> j) & 1ull) ? 0.5 : -0.5;
        d += J * Delta * szi * szj;
    }
    for (int i = 0; i < L; ++i) d += h[i] * (((s >> i) & 1ull) ? 0.5 : -0.5);
    return d;
}

/* Fill CSR arrays (rowptr[D+1], col[nnz], val[nnz]).  Returns 0, or -1 if a flipped
 * state is not found in the basis (which cannot happen for a correct basis). */
int orc_ham_csr(int L, const uint64_t *basis, int64_t D, double J, double Delta,
                const double *h, int pbc, int64_t *rowptr, int64_t *col, double *val)
{
    int nb = n_bonds(L, pbc);
    int64_t k = 0;
    rowptr[0] = 0;
    for (int64_t r = 0; r < D; ++r) {
        uint64_t s = basis[r];
        col[k] = r;
        val[k] = orc_diag(s, L, J, Delta, h, pbc);
        ++k;
        for (int b = 0; b < nb; ++b) {
            int i, j;
            bond_sites(b, L, &i, &j);
            if (((s >> i) & 1ull) == ((s >> j) & 1ull)) continue;
            uint64_t s2 = s ^ ((1ull << i) | (1ull << j));   /* hop across the bond */
            int64_t c = orc_lookup(basis, D, s2);
            if (c < 0) return -1;
            col[k] = c;
            val[k] = 0.5 * J;
            ++k;
        }
        rowptr[r + 1] = k;
    }
    return 0;
}

/* y = A x for a real CSR matrix and complex vectors stored as interleaved (re, im). */
void orc_spmv(int64_t D, const int64_t *rowptr, const int64_t *col, const double *val,
              const double *x, double *y)
{
    for (int64_t r = 0; r < D; ++r) {
        double re = 0.0, im = 0.0;
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
            re += val[k] * x[2 * col[k]];
            im += val[k] * x[2 * col[k] + 1];
        }
        y[2 * r] = re;
        y[2 * r + 1] = im;
    }
}
