/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU statement of what the GPU library
 * computes: the exact S lowest (energy, configuration) pairs of an Ising
 * instance by exhaustive enumeration.  Only tests/, __graft_entry__.smoke()
 * and the cpu_baseline / reference leg of bench.py may load or call it.  It
 * shares no code, table or helper with the CUDA library and must never be
 * reached from the product path.
 *
 * Definitions followed (Jalowiecki, Rams, Gardas, "Brute-forcing spin-glass
 * problems with CUDA"):
 *   - Energy, Sec. 2, Eq. (1): a pair sum over the edges of the graph plus a
 *     field sum.  The library fixes the overall sign to
 *         E(s) = + sum_{i<j} J_ij s_i s_j + sum_i h_i s_i ,
 *     i.e. the paper's H with J and h negated.  J is a dense row-major
 *     n x n matrix of which only the strict upper triangle (i < j) is read;
 *     the diagonal and the lower triangle are ignored.
 *   - Encoding, Sec. 3, Eqs. (4)-(5): a configuration is the integer whose
 *     binary digits are q = (s + 1) / 2.  Reading fixed by the library: bit i
 *     of c (least significant bit = spin 0) is q_i, so s_i = +1 iff bit i = 1.
 *   - Chunk offset, Sec. 3, Eq. (6): configuration = offset + index; the
 *     subspace mode below fixes the top `fixed_bits` bits of c (the offset)
 *     and enumerates the rest.
 *   - Algorithm 1 (Sec. 3): the output is the S lowest configurations sorted
 *     by energy.  The library orders ties by the configuration integer, so
 *     the result is the first S records under the total order (E, c).
 *   - QUBO form, Sec. 2, Eq. (2), with the same overall sign flip:
 *         F(q) = + sum_{i<j} a_ij q_i q_j + sum_i b_i q_i ,
 *     q_i = bit i of c (the binary digits of Eq. (4)); strict upper triangle
 *     of a read, like J.
 *   - q-state Potts model (Sec. 2: the extension to other classical
 *     spin-glass models), same sign convention:
 *         E(sigma) = sum_{i<j} J_ij [sigma_i == sigma_j] + sum_i h_i(sigma_i),
 *     sigma_i = base-q digit i of c, h stored as h[i*q + v].
 *   - Gradient of L = sum_k g_k E(s^(k)) with respect to J_ij (i<j) and h_i,
 *     which follows from Eq. (1) being linear in J and h:
 *         dL/dJ_ij = sum_k g_k s_i^(k) s_j^(k),   dL/dh_i = sum_k g_k s_i^(k).
 *
 * Arithmetic: float instances in FP64, integer instances in int64, by the
 * direct double loop (pairs first in (i, j) order, then fields).  Selection
 * uses the C library's qsort as the sorting step: either all records of the
 * enumerated range are materialised and sorted, or each OpenMP thread keeps a
 * bounded max-heap of its S best records and the union is sorted at the end.
 *
 * Compile-time switch ORACLE_PLANT=k plants one deliberate mistake; it exists
 * only so the tests can show that the pins catch that class of error.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

/* spin value s_i in {-1, +1} of configuration c (Sec. 3, Eqs. (4)-(5)) */
static int spin_of(uint64_t c, int i, int n)
{
#if ORACLE_PLANT == 5
    i = n - 1 - i;                     /* planted: reversed bit order */
#else
    (void)n;
#endif
    int bit = (int)((c >> i) & 1u);
#if ORACLE_PLANT == 6
    return bit ? -1 : +1;              /* planted: inverted spin mapping */
#else
    return bit ? +1 : -1;
#endif
}

static double coupling_f64(const double *J, int n, int i, int j)
{
#if ORACLE_PLANT == 3
    return J[(size_t)j * n + i];       /* planted: lower triangle read */
#else
    return J[(size_t)i * n + j];
#endif
}

static int32_t coupling_i32(const int32_t *J, int n, int i, int j)
{
#if ORACLE_PLANT == 3
    return J[(size_t)j * n + i];
#else
    return J[(size_t)i * n + j];
#endif
}

/* first partner index of the pair loop: j = i + 1 (strict upper triangle) */
static int pair_start(int i)
{
#if ORACLE_PLANT == 4
    return i;                          /* planted: diagonal included */
#else
    return i + 1;
#endif
}

/* Sec. 2, Eq. (1), sign fixed as E = +sum J s s + sum h s, FP64 */
double oracle_energy_f64(int n, const double *J, const double *h, uint64_t c)
{
#if ORACLE_PLANT == 10
    float pair = 0.0f, field = 0.0f;   /* planted: single precision */
#else
    double pair = 0.0, field = 0.0;
#endif
    for (int i = 0; i < n; i++) {
        int si = spin_of(c, i, n);
        for (int j = pair_start(i); j < n; j++) {
            int sj = spin_of(c, j, n);
            pair += coupling_f64(J, n, i, j) * (double)(si * sj);
        }
    }
    for (int i = 0; i < n; i++)
        field += h[i] * (double)spin_of(c, i, n);
#if ORACLE_PLANT == 1
    field = 0.0;                        /* planted: field term dropped */
#endif
#if ORACLE_PLANT == 2
    return -(double)pair + (double)field; /* planted: pair sign flipped */
#else
    return (double)pair + (double)field;
#endif
}

/* Sec. 2, Eq. (1) for integer couplings and fields, exact in int64 */
int64_t oracle_energy_i64(int n, const int32_t *J, const int32_t *h, uint64_t c)
{
    int64_t pair = 0, field = 0;
    for (int i = 0; i < n; i++) {
        int si = spin_of(c, i, n);
        for (int j = pair_start(i); j < n; j++) {
            int sj = spin_of(c, j, n);
            pair += (int64_t)coupling_i32(J, n, i, j) * (int64_t)(si * sj);
        }
    }
    for (int i = 0; i < n; i++)
        field += (int64_t)h[i] * (int64_t)spin_of(c, i, n);
#if ORACLE_PLANT == 1
    field = 0;
#endif
#if ORACLE_PLANT == 2
    return -pair + field;
#else
    return pair + field;
#endif
}

/* binary variable q_i of configuration c (Sec. 3, Eq. (4)) */
static int binary_of(uint64_t c, int i)
{
    return (int)((c >> i) & 1u);
}

/* first partner index j of row i in the QUBO pair sum (strict upper triangle) */
static int qubo_pair_start(int i)
{
#if ORACLE_PLANT == 11
    return i;                          /* planted: diagonal a_ii q_i q_i included */
#else
    return i + 1;
#endif
}

/* coupling a_ij, i < j, of a row-major matrix */
static double qubo_coupling_f64(const double *a, int n, int i, int j)
{
#if ORACLE_PLANT == 12
    return a[j * n + i];               /* planted: lower triangle read */
#else
    return a[i * n + j];
#endif
}

/* Sec. 2, Eq. (2) with the overall sign flipped, FP64 */
double oracle_qubo_energy_f64(int n, const double *a, const double *b, uint64_t c)
{
    double pair = 0.0, field = 0.0;
    for (int i = 0; i < n; i++) {
        if (!binary_of(c, i)) continue;
        for (int j = qubo_pair_start(i); j < n; j++)
            if (binary_of(c, j)) pair += qubo_coupling_f64(a, n, i, j);
    }
    for (int i = 0; i < n; i++)
        if (binary_of(c, i)) field += b[i];
    return pair + field;
}

/* Sec. 2, Eq. (2) for integer coefficients, exact in int64 */
int64_t oracle_qubo_energy_i64(int n, const int32_t *a, const int32_t *b, uint64_t c)
{
    int64_t pair = 0, field = 0;
    for (int i = 0; i < n; i++) {
        if (!binary_of(c, i)) continue;
        for (int j = qubo_pair_start(i); j < n; j++)
#if ORACLE_PLANT == 12
            if (binary_of(c, j)) pair += a[j * n + i];
#else
            if (binary_of(c, j)) pair += a[i * n + j];
#endif
    }
    for (int i = 0; i < n; i++)
        if (binary_of(c, i)) field += b[i];
    return pair + field;
}

/* base-q digit i of configuration c (generalising Sec. 3, Eq. (4)) */
static int digit_of(uint64_t c, int i, int q)
{
    for (int k = 0; k < i; k++) c /= (uint64_t)q;
    return (int)(c % (uint64_t)q);
}

/* the indicator [sigma_i == sigma_j] of the Potts pair term */
static int same_state(int a, int b)
{
#if ORACLE_PLANT == 13
    return a != b;                     /* planted: inequality */
#else
    return a == b;
#endif
}

/* field h_i(v) of a row-major n x q table */
static double potts_field_f64(const double *h, int n, int q, int i, int v)
{
#if ORACLE_PLANT == 14
    (void)q;
    return h[v * n + i];               /* planted: transposed field table */
#else
    (void)n;
    return h[i * q + v];
#endif
}

/* q-state Potts energy, FP64 */
double oracle_potts_energy_f64(int n, int q, const double *J, const double *h, uint64_t c)
{
    double pair = 0.0, field = 0.0;
    for (int i = 0; i < n; i++) {
        int di = digit_of(c, i, q);
        for (int j = i + 1; j < n; j++)
            if (same_state(di, digit_of(c, j, q))) pair += J[i * n + j];
        field += potts_field_f64(h, n, q, i, di);
    }
    return pair + field;
}

/* q-state Potts energy, integer coefficients, exact in int64 */
int64_t oracle_potts_energy_i64(int n, int q, const int32_t *J, const int32_t *h, uint64_t c)
{
    int64_t pair = 0, field = 0;
    for (int i = 0; i < n; i++) {
        int di = digit_of(c, i, q);
        for (int j = i + 1; j < n; j++)
            if (same_state(di, digit_of(c, j, q))) pair += J[i * n + j];
#if ORACLE_PLANT == 14
        field += h[di * n + i];
#else
        field += h[i * q + di];
#endif
    }
    return pair + field;
}

/* ---- selection: first S records under the total order (E, c) ---------- */

typedef struct {
    double e;      /* energy of a float instance */
    int64_t ie;    /* energy of an integer instance */
    uint64_t c;    /* configuration integer */
} rec_t;

static int g_is_int; /* set before each selection; read-only while sorting */
static int g_qubo;   /* 0: Ising energy of Eq. (1), 1: QUBO value of Eq. (2), 2: Potts energy */
static int g_potts_q; /* number of Potts states (model 2) */

static int rec_less(const rec_t *a, const rec_t *b)
{
    if (g_is_int) {
        if (a->ie != b->ie) return a->ie < b->ie;
    } else {
        if (a->e != b->e) return a->e < b->e;
    }
#if ORACLE_PLANT == 7
    return a->c > b->c;                 /* planted: ties by descending c */
#else
    return a->c < b->c;
#endif
}

static int rec_cmp(const void *pa, const void *pb)
{
    const rec_t *a = (const rec_t *)pa, *b = (const rec_t *)pb;
    if (rec_less(a, b)) return -1;
    if (rec_less(b, a)) return 1;
    return 0;
}

/* bounded max-heap of the `cap` smallest records seen so far */
static void heap_push(rec_t *heap, int *size, int cap, rec_t r)
{
    if (*size < cap) {
        int k = (*size)++;
        heap[k] = r;
        while (k > 0) {                 /* sift up: parent must be >= child */
            int p = (k - 1) / 2;
            if (!rec_less(&heap[p], &heap[k])) break;
            rec_t t = heap[p]; heap[p] = heap[k]; heap[k] = t;
            k = p;
        }
        return;
    }
    if (!rec_less(&r, &heap[0])) return; /* not better than the worst kept */
    heap[0] = r;
    int k = 0;
    for (;;) {                          /* sift down */
        int l = 2 * k + 1, rr = l + 1, m = k;
        if (l < cap && rec_less(&heap[m], &heap[l])) m = l;
        if (rr < cap && rec_less(&heap[m], &heap[rr])) m = rr;
        if (m == k) break;
        rec_t t = heap[m]; heap[m] = heap[k]; heap[k] = t;
        k = m;
    }
}

static rec_t make_rec(int n, const void *J, const void *h, uint64_t c)
{
    rec_t r;
    r.c = c;
    if (g_is_int) {
        if (g_qubo == 2) r.ie = oracle_potts_energy_i64(n, g_potts_q, (const int32_t *)J, (const int32_t *)h, c);
        else if (g_qubo == 1) r.ie = oracle_qubo_energy_i64(n, (const int32_t *)J, (const int32_t *)h, c);
        else r.ie = oracle_energy_i64(n, (const int32_t *)J, (const int32_t *)h, c);
        r.e = (double)r.ie;
    } else {
        if (g_qubo == 2) r.e = oracle_potts_energy_f64(n, g_potts_q, (const double *)J, (const double *)h, c);
        else if (g_qubo == 1) r.e = oracle_qubo_energy_f64(n, (const double *)J, (const double *)h, c);
        else r.e = oracle_energy_f64(n, (const double *)J, (const double *)h, c);
        r.ie = 0;
    }
    return r;
}

#define FULL_SORT_LIMIT ((uint64_t)1 << 22)

/*
 * Enumerate c = (fixed_value << (n - fixed_bits)) + x for every
 * x in [0, 2^(n - fixed_bits)) (Sec. 3, Eq. (6): offset + index) and return
 * the S lowest records.  mode: 0 = automatic, 1 = materialise and sort all,
 * 2 = per-thread bounded heaps.  threads <= 0 uses the OpenMP default.
 * Returns 0 on success, -1 on invalid arguments, -2 when memory is short.
 */
static int low_spectrum(int is_int, int qubo, int n, const void *J, const void *h, int S,
                        int fixed_bits, uint64_t fixed_value, int mode, int threads,
                        rec_t *out)
{
    g_qubo = qubo;
    if (n < 1 || n > 64 || S < 1 || fixed_bits < 0 || fixed_bits > n) return -1;
    int free_bits = n - fixed_bits;
    if (free_bits > 62) return -1;
    uint64_t count = (uint64_t)1 << free_bits;
    if (qubo == 2) {                   /* Potts: all q^n configurations, no fixed digits */
        if (fixed_bits != 0 || g_potts_q < 2) return -1;
        count = 1;
        for (int i = 0; i < n; i++) {
            if (count > ((uint64_t)1 << 62) / (uint64_t)g_potts_q) return -1;
            count *= (uint64_t)g_potts_q;
        }
    }
    if ((uint64_t)S > count) return -1;
    if (fixed_bits > 0 && fixed_bits < 64 && (fixed_value >> fixed_bits) != 0) return -1;
    uint64_t base = fixed_bits ? (fixed_value << free_bits) : 0;
    g_is_int = is_int;
    if (mode == 0) mode = (count <= FULL_SORT_LIMIT) ? 1 : 2;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif

    if (mode == 1) {
        if (count > FULL_SORT_LIMIT) return -1;
        rec_t *all = (rec_t *)malloc(sizeof(rec_t) * (size_t)count);
        if (!all) return -2;
        int64_t cnt = (int64_t)count;
#pragma omp parallel for schedule(static)
        for (int64_t x = 0; x < cnt; x++)
            all[x] = make_rec(n, J, h, base + (uint64_t)x);
        qsort(all, (size_t)count, sizeof(rec_t), rec_cmp);
#if ORACLE_PLANT == 8
        memcpy(out, all + 1, sizeof(rec_t) * (size_t)(S - 1)); /* planted: first record lost */
        out[S - 1] = all[S < (int)count ? S : 0];
#else
        memcpy(out, all, sizeof(rec_t) * (size_t)S);
#endif
        free(all);
        return 0;
    }

    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    rec_t *heaps = (rec_t *)malloc(sizeof(rec_t) * (size_t)S * (size_t)nt);
    int *sizes = (int *)calloc((size_t)nt, sizeof(int));
    if (!heaps || !sizes) { free(heaps); free(sizes); return -2; }
    int64_t cnt = (int64_t)count;
#pragma omp parallel num_threads(nt)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        rec_t *heap = heaps + (size_t)t * S;
#pragma omp for schedule(static)
        for (int64_t x = 0; x < cnt; x++)
            heap_push(heap, &sizes[t], S, make_rec(n, J, h, base + (uint64_t)x));
    }
    /* union of the per-thread heaps, then one sort */
    size_t total = 0;
    for (int t = 0; t < nt; t++) total += (size_t)sizes[t];
    rec_t *all = (rec_t *)malloc(sizeof(rec_t) * (total ? total : 1));
    if (!all) { free(heaps); free(sizes); return -2; }
    size_t k = 0;
    for (int t = 0; t < nt; t++)
        for (int i = 0; i < sizes[t]; i++) all[k++] = heaps[(size_t)t * S + i];
    qsort(all, total, sizeof(rec_t), rec_cmp);
#if ORACLE_PLANT == 8
    memcpy(out, all + 1, sizeof(rec_t) * (size_t)(S - 1));
    out[S - 1] = all[0];
#else
    memcpy(out, all, sizeof(rec_t) * (size_t)S);
#endif
    free(all); free(heaps); free(sizes);
    return 0;
}

int oracle_low_spectrum_f64(int n, const double *J, const double *h, int S,
                            int fixed_bits, uint64_t fixed_value, int mode, int threads,
                            double *out_e, uint64_t *out_c)
{
    if (S < 1) return -1;
    rec_t *out = (rec_t *)malloc(sizeof(rec_t) * (size_t)S);
    if (!out) return -2;
    int rc = low_spectrum(0, 0, n, J, h, S, fixed_bits, fixed_value, mode, threads, out);
    if (rc == 0)
        for (int k = 0; k < S; k++) { out_e[k] = out[k].e; out_c[k] = out[k].c; }
    free(out);
    return rc;
}

int oracle_low_spectrum_i64(int n, const int32_t *J, const int32_t *h, int S,
                            int fixed_bits, uint64_t fixed_value, int mode, int threads,
                            int64_t *out_e, uint64_t *out_c)
{
    if (S < 1) return -1;
    rec_t *out = (rec_t *)malloc(sizeof(rec_t) * (size_t)S);
    if (!out) return -2;
    int rc = low_spectrum(1, 0, n, J, h, S, fixed_bits, fixed_value, mode, threads, out);
    if (rc == 0)
        for (int k = 0; k < S; k++) { out_e[k] = out[k].ie; out_c[k] = out[k].c; }
    free(out);
    return rc;
}

/* The S lowest (E, c) of the q-state Potts model, FP64 */
int oracle_potts_low_spectrum_f64(int n, int q, const double *J, const double *h, int S, int mode, int threads,
                                  double *out_e, uint64_t *out_c)
{
    if (S < 1 || q < 2 || q > 255) return -1;
    rec_t *out = (rec_t *)malloc(sizeof(rec_t) * (size_t)S);
    if (!out) return -2;
    g_potts_q = q;
    int rc = low_spectrum(0, 2, n, J, h, S, 0, 0, mode, threads, out);
    if (rc == 0)
        for (int k = 0; k < S; k++) { out_e[k] = out[k].e; out_c[k] = out[k].c; }
    free(out);
    return rc;
}

/* The S lowest (E, c) of the q-state Potts model, integer coefficients, exact */
int oracle_potts_low_spectrum_i64(int n, int q, const int32_t *J, const int32_t *h, int S, int mode, int threads,
                                  int64_t *out_e, uint64_t *out_c)
{
    if (S < 1 || q < 2 || q > 255) return -1;
    rec_t *out = (rec_t *)malloc(sizeof(rec_t) * (size_t)S);
    if (!out) return -2;
    g_potts_q = q;
    int rc = low_spectrum(1, 2, n, J, h, S, 0, 0, mode, threads, out);
    if (rc == 0)
        for (int k = 0; k < S; k++) { out_e[k] = out[k].ie; out_c[k] = out[k].c; }
    free(out);
    return rc;
}

/* The S lowest (F, c) of the QUBO form (Sec. 2, Eq. (2)), FP64 */
int oracle_qubo_low_spectrum_f64(int n, const double *a, const double *b, int S,
                                 int fixed_bits, uint64_t fixed_value, int mode, int threads,
                                 double *out_f, uint64_t *out_c)
{
    if (S < 1) return -1;
    rec_t *out = (rec_t *)malloc(sizeof(rec_t) * (size_t)S);
    if (!out) return -2;
    int rc = low_spectrum(0, 1, n, a, b, S, fixed_bits, fixed_value, mode, threads, out);
    if (rc == 0)
        for (int k = 0; k < S; k++) { out_f[k] = out[k].e; out_c[k] = out[k].c; }
    free(out);
    return rc;
}

/* The S lowest (F, c) of the QUBO form for integer coefficients, exact */
int oracle_qubo_low_spectrum_i64(int n, const int32_t *a, const int32_t *b, int S,
                                 int fixed_bits, uint64_t fixed_value, int mode, int threads,
                                 int64_t *out_f, uint64_t *out_c)
{
    if (S < 1) return -1;
    rec_t *out = (rec_t *)malloc(sizeof(rec_t) * (size_t)S);
    if (!out) return -2;
    int rc = low_spectrum(1, 1, n, a, b, S, fixed_bits, fixed_value, mode, threads, out);
    if (rc == 0)
        for (int k = 0; k < S; k++) { out_f[k] = out[k].ie; out_c[k] = out[k].c; }
    free(out);
    return rc;
}

/* Energies of all 2^n configurations in increasing c (n <= 26), Eq. (1). */
int oracle_all_energies_f64(int n, const double *J, const double *h, double *out)
{
    if (n < 1 || n > 26) return -1;
    int64_t cnt = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < cnt; c++)
        out[c] = oracle_energy_f64(n, J, h, (uint64_t)c);
    return 0;
}

int oracle_all_energies_i64(int n, const int32_t *J, const int32_t *h, int64_t *out)
{
    if (n < 1 || n > 26) return -1;
    int64_t cnt = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < cnt; c++)
        out[c] = oracle_energy_i64(n, J, h, (uint64_t)c);
    return 0;
}

/*
 * Gradient of L = sum_b sum_k g[b,k] E_b(s^(b,k)) with respect to the strict
 * upper triangle of each J_b and to each h_b (linearity of Eq. (1)).
 * Instance b has n[b] spins; its dense n x n block of dJ starts at
 * J_off[b] and its field gradient at h_off[b].  Entries on or below the
 * diagonal are written as zero.  states and g are B x S row-major.
 */
int oracle_grad(int B, const int *n, int S, const uint64_t *states, const double *g,
                const int64_t *J_off, const int64_t *h_off, double *dJ, double *dh)
{
    for (int b = 0; b < B; b++) {
        int nb = n[b];
        if (nb < 1 || nb > 64) return -1;
        double *dJb = dJ + J_off[b];
        double *dhb = dh + h_off[b];
        for (int i = 0; i < nb; i++) {
            dhb[i] = 0.0;
            for (int j = 0; j < nb; j++) dJb[(size_t)i * nb + j] = 0.0;
        }
        for (int k = 0; k < S; k++) {
            uint64_t c = states[(size_t)b * S + k];
            double w = g[(size_t)b * S + k];
            for (int i = 0; i < nb; i++) {
                int si = spin_of(c, i, nb);
                for (int j = i + 1; j < nb; j++) {
#if ORACLE_PLANT == 9
                    dJb[(size_t)i * nb + j] += w * (double)si;   /* planted: s_j dropped */
#else
                    dJb[(size_t)i * nb + j] += w * (double)(si * spin_of(c, j, nb));
#endif
                }
                dhb[i] += w * (double)si;
            }
        }
    }
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int oracle_plant(void) { return ORACLE_PLANT; }
