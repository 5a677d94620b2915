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

/* ------------------------------------------------------------------ early-time moments
 *
 * The return amplitude of Eq. SP for a basis state s0, A(t) = <s0| exp(-iHt) |s0>, is the
 * power series  sum_n (-it)^n mu_n / n!  in the moments mu_n = <s0| (H - c)^n |s0> of the
 * shifted Hamiltonian (c = the diagonal element of s0; the shift multiplies A by a phase
 * and leaves P unchanged).  v_k = (H - c)^k |s0> has its support on the states that k hops
 * or fewer lead to from s0 (a hop exchanges the two sites of an antiparallel bond), so
 *     mu_{2k} = <v_k, v_k>,   mu_{2k+1} = <v_k, v_{k+1}>
 * for k < K need only the states within K hops of s0 ("the ball"), not the whole sector.
 */

static int cmp_u64(const void *a, const void *b)
{
    const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Sort a[0..n) and drop repeats; returns the new length. */
static int64_t sort_unique(uint64_t *a, int64_t n)
{
    if (n == 0) return 0;
    qsort(a, (size_t)n, sizeof(uint64_t), cmp_u64);
    int64_t k = 1;
    for (int64_t i = 1; i < n; ++i)
        if (a[i] != a[k - 1]) a[k++] = a[i];
    return k;
}

/* mu[0..2K] for s0 and the number of states in its K-hop ball (*nball).  Returns 0, -1 on
 * bad arguments or an allocation failure, -2 if a hopped state is missing from the ball
 * (which cannot happen when the ball is built correctly). */
int orc_moments(int L, double J, double Delta, const double *h, int pbc, uint64_t s0, int K,
                double *mu, int64_t *nball)
{
    if (L < 1 || L > 62 || K < 0 || K > 64 || (L < 64 && (s0 >> L) != 0ull)) return -1;
    const int nb = n_bonds(L, pbc);
    uint64_t *all = (uint64_t *)malloc(sizeof(uint64_t)), *front = (uint64_t *)malloc(sizeof(uint64_t));
    if (!all || !front) { free(all); free(front); return -1; }
    all[0] = front[0] = s0;
    int64_t nall = 1, nfront = 1;
    for (int k = 1; k <= K; ++k) {
        /* every state one hop away from the previous level, without repeats */
        uint64_t *gen = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nfront * (nb > 0 ? nb : 1)));
        if (!gen) { free(all); free(front); return -1; }
        int64_t ng = 0;
        for (int64_t q = 0; q < nfront; ++q) {
            const uint64_t s = front[q];
            for (int b = 0; b < nb; ++b) {
                int i, j;
                bond_sites(b, L, &i, &j);
                if (((s >> i) & 1ull) != ((s >> j) & 1ull)) gen[ng++] = s ^ ((1ull << i) | (1ull << j));
            }
        }
        ng = sort_unique(gen, ng);
        /* the new level: generated states not yet in the ball (both lists ascending) */
        uint64_t *nw = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(ng > 0 ? ng : 1));
        uint64_t *merged = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nall + ng));
        if (!nw || !merged) { free(gen); free(nw); free(merged); free(all); free(front); return -1; }
        int64_t nn = 0, a = 0, g = 0, m = 0;
        while (g < ng) {
            if (a < nall && all[a] < gen[g]) { merged[m++] = all[a++]; continue; }
            if (a < nall && all[a] == gen[g]) { merged[m++] = all[a++]; ++g; continue; }
            nw[nn++] = gen[g];
            merged[m++] = gen[g++];
        }
        while (a < nall) merged[m++] = all[a++];
        free(gen);
        free(all);
        free(front);
        all = merged;
        nall = m;
        front = nw;
        nfront = nn;
    }
    free(front);
    *nball = nall;
    double *v = (double *)calloc((size_t)nall, sizeof(double));
    double *w = (double *)calloc((size_t)nall, sizeof(double));
    if (!v || !w) { free(v); free(w); free(all); return -1; }
    const double c = orc_diag(s0, L, J, Delta, h, pbc);
    v[orc_lookup(all, nall, s0)] = 1.0;
    int rc = 0;
    for (int k = 0; k <= K && rc == 0; ++k) {
        double nv = 0.0;
        for (int64_t r = 0; r < nall; ++r) nv += v[r] * v[r];
        mu[2 * k] = nv;
        if (k == K) break;
        /* w = (H - c) v, pushed from the entries of v (all inside the (K-1)-hop ball) */
        for (int64_t r = 0; r < nall; ++r) w[r] = 0.0;
        for (int64_t r = 0; r < nall && rc == 0; ++r) {
            if (v[r] == 0.0) continue;
            const uint64_t s = all[r];
            w[r] += (orc_diag(s, L, J, Delta, h, pbc) - c) * v[r];
            for (int b = 0; b < nb; ++b) {
                int i, j;
                bond_sites(b, L, &i, &j);
                if (((s >> i) & 1ull) == ((s >> j) & 1ull)) continue;
                const int64_t q = orc_lookup(all, nall, s ^ ((1ull << i) | (1ull << j)));
                if (q < 0) { rc = -2; break; }
                w[q] += 0.5 * J * v[r];
            }
        }
        double vw = 0.0;
        for (int64_t r = 0; r < nall; ++r) vw += v[r] * w[r];
        mu[2 * k + 1] = vw;
        double *tmp = v;
        v = w;
        w = tmp;
    }
    free(v);
    free(w);
    free(all);
    return rc;
}
