/*
 * CPU oracle for the semiring product and closure of de Bondt, "Fast algorithms
 * for anti-distance matrices as a generalization of Boolean matrices"
 * (arXiv 1705.08743).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: it exists so that tests, the smoke check and the CPU baseline of
 * the benchmark can check the CUDA kernels against plain, slow, obviously
 * correct code.  It shares no code, header, table or helper with the CUDA path.
 *
 * Entries are unsigned integers in S·D = {0, 1, ..., S} (Section 4, where the
 * paper scales D = {0, 1/S, ..., 1} by S).  S = 1 is the Boolean set B = {0,1}
 * of Section 2.  Every array here is row-major and dense (no padding) unless a
 * leading dimension is given.
 *
 *   a ⊕ b = max(a, b)                          (Section 2, "∨"; Section 3 keeps it)
 *   a ⊗ b = min(a, b)            for S = 1     (Section 2, "∧")
 *   a ⊗ b = max(a + b − S, 0)    for S > 1     (Section 3, the definition on D,
 *                                               scaled by S as in Section 4)
 *
 * Readings of the paper taken here:
 *  - A_ij = 1 (or > 0) means an edge i -> j, and (A ⊗ B)_ij = ⊕_k A_ik ⊗ B_kj
 *    exactly as in the formula of Section 2; the sentence after it that names
 *    "a B-edge from i to k and an A-edge from k to j" is read as a slip.
 *  - The closure is the non-reflexive one, A ⊕ A⊗A ⊕ ... (Section 2, "trcl"):
 *    T_ii is the best cycle through i.
 *  - Saturation: a path whose length (sum of S − a over its edges) is >= S has
 *    value 0, i.e. exactly max(S − length, 0).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;

/* ⊗ on {0..S}: Section 2 (S = 1) and Section 3 (S > 1).  64-bit sum: no overflow. */
static inline uint32_t sr_times(uint32_t a, uint32_t b, uint32_t S)
{
    if (S == 1)
        return a < b ? a : b;
    uint64_t s = (uint64_t)a + (uint64_t)b;
    return s > (uint64_t)S ? (uint32_t)(s - S) : 0u;
}

static inline uint32_t sr_plus(uint32_t a, uint32_t b) { return a > b ? a : b; }

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * Product P = (accumulate ? C : 0) ⊕ A ⊗ B, written into C (Section 2, the
 * column-times-row form "P := P ∨ (A_col k ⊗ B_row k)" for k = 1..C, and the
 * Section 4 listings, which run k from the last column down and skip zero
 * entries of A because 0 ⊗ b = 0).  A is R×K, B is K×N, C is R×N.
 * Rows of P are independent, so blocks of rows run on separate threads; inside
 * a block the loop order is the paper's.
 */
void or_mul(const uint32_t *A, const uint32_t *B, uint32_t *C,
            i64 R, i64 K, i64 N, uint32_t S, int accumulate)
{
    if (!accumulate)
        memset(C, 0, (size_t)(R * N) * sizeof(uint32_t));
    const i64 RB = 16;
#pragma omp parallel for schedule(dynamic, 1)
    for (i64 r0 = 0; r0 < R; r0 += RB) {
        i64 r1 = r0 + RB < R ? r0 + RB : R;
        for (i64 k = K - 1; k >= 0; --k) {
            const uint32_t *Bk = B + k * N;               /* row k of B */
            for (i64 r = r0; r < r1; ++r) {
                uint32_t a = A[r * K + k];                /* entry (r, k) of A */
                if (a == 0)
                    continue;
                uint32_t *Cr = C + r * N;                 /* row r of P */
                if (S == 1) {
                    for (i64 j = 0; j < N; ++j)
                        Cr[j] = sr_plus(Cr[j], sr_times(a, Bk[j], 1));
                } else {
                    for (i64 j = 0; j < N; ++j)
                        Cr[j] = sr_plus(Cr[j], sr_times(a, Bk[j], S));
                }
            }
        }
    }
}

/*
 * The product by its formula, entry by entry: P_ij = ⊕_k A_ik ⊗ B_kj (Section 2).
 * Only for sampled entries: O(K) per entry.
 */
uint32_t or_mul_entry(const uint32_t *A, const uint32_t *B, i64 K, i64 N,
                      i64 i, i64 j, uint32_t S)
{
    uint32_t p = 0;
    for (i64 k = 0; k < K; ++k)
        p = sr_plus(p, sr_times(A[i * K + k], B[k * N + j], S));
    return p;
}

/*
 * Warshall's algorithm (Section 2) and its Floyd generalisation (Section 3):
 *   T := A;  for k = 1..D:  T := T ⊕ (T_col k ⊗ T_row k),  in place.
 * During step k, row k and column k do not change: T_kk ⊗ x <= x for every
 * entry x (min(T_kk, x) <= x; max(T_kk + x − S, 0) <= x as T_kk <= S), so the
 * rows i != k of step k are independent and may run on separate threads.
 */
void or_warshall(uint32_t *T, i64 D, uint32_t S)
{
    for (i64 k = 0; k < D; ++k) {
        const uint32_t *Tk = T + k * D;
#pragma omp parallel for schedule(static)
        for (i64 i = 0; i < D; ++i) {
            if (i == k)
                continue;
            uint32_t a = T[i * D + k];
            if (a == 0)
                continue;
            uint32_t *Ti = T + i * D;
            for (i64 j = 0; j < D; ++j)
                Ti[j] = sr_plus(Ti[j], sr_times(a, Tk[j], S));
        }
    }
}

/*
 * Closure by repeated squaring (Section 2): for every D' >= D,
 *   A ⊕ A^2 ⊕ ... ⊕ A^D' = A ⊗ (I ⊕ A)^(D'−1).
 * With m = ceil(log2(max(D−1, 1))) squarings, (I ⊕ A)^(2^m) has 2^m >= D−1.
 * I has S on the diagonal (S ⊗ b = b) and 0 elsewhere.  work holds 2·D·D entries.
 */
void or_closure_squaring(const uint32_t *A, uint32_t *T, i64 D, uint32_t S, uint32_t *work)
{
    uint32_t *M = work, *M2 = work + D * D;
    memcpy(M, A, (size_t)(D * D) * sizeof(uint32_t));
    for (i64 i = 0; i < D; ++i)
        M[i * D + i] = S;                                   /* I ⊕ A */
    int m = 0;
    while (((i64)1 << m) < (D - 1 > 1 ? D - 1 : 1))
        ++m;
    for (int s = 0; s < m; ++s) {
        or_mul(M, M, M2, D, D, D, S, 0);
        uint32_t *t = M; M = M2; M2 = t;
    }
    or_mul(A, M, T, D, D, D, S, 0);
}

/*
 * Row src of the closure by its graph reading (Sections 2 and 3): entry j is
 * the best value of a path src -> j with at least one edge, where an entry
 * a > 0 is an edge of length S − a and a path of length L has value
 * max(S − L, 0).  Shortest lengths by Dijkstra's method (non-negative integer
 * lengths, array scan, O(D^2)).  For S = 1 this is plain reachability.
 */
void or_closure_row(const uint32_t *A, i64 D, uint32_t S, i64 src, uint32_t *row)
{
    const i64 INF = INT64_MAX / 4;
    i64 *dist = (i64 *)malloc((size_t)D * sizeof(i64));
    char *done = (char *)calloc((size_t)D, 1);
    for (i64 v = 0; v < D; ++v) {
        uint32_t a = A[src * D + v];
        dist[v] = a ? (i64)(S - a) : INF;                 /* one-edge paths */
    }
    for (;;) {
        i64 u = -1, best = INF;
        for (i64 v = 0; v < D; ++v)
            if (!done[v] && dist[v] < best) { best = dist[v]; u = v; }
        if (u < 0)
            break;
        done[u] = 1;
        for (i64 v = 0; v < D; ++v) {
            uint32_t a = A[u * D + v];
            if (a && dist[u] + (i64)(S - a) < dist[v])
                dist[v] = dist[u] + (i64)(S - a);
        }
    }
    for (i64 v = 0; v < D; ++v)
        row[v] = dist[v] >= (i64)S ? 0u : (uint32_t)((i64)S - dist[v]);
    free(dist);
    free(done);
}

/* ------------------------------------------------------------------------ */
/* Boolean matrices on 64-bit words (Section 4, matBool)                      */
/* ------------------------------------------------------------------------ */

/*
 * Entry (r, c) of a bit matrix stored as rows of 64-bit blocks: bit (c & 7) of
 * byte (c >> 3) of row r, as in the matBool listing of Section 4.
 */
static inline int bit_get(const uint64_t *M, i64 ldw, i64 r, i64 c)
{
    const unsigned char *row = (const unsigned char *)(M + r * ldw);
    return (row[c >> 3] >> (c & 7)) & 1;
}

static inline void bit_set(uint64_t *M, i64 ldw, i64 r, i64 c)
{
    unsigned char *row = (unsigned char *)(M + r * ldw);
    row[c >> 3] |= (unsigned char)(1u << (c & 7));
}

/* Dense 0/1 bytes (R×C, row-major) -> bit rows of ldw 64-bit words, pad bits 0. */
void or_pack_bits(const uint8_t *dense, i64 R, i64 C, uint64_t *M, i64 ldw)
{
    memset(M, 0, (size_t)(R * ldw) * sizeof(uint64_t));
    for (i64 r = 0; r < R; ++r)
        for (i64 c = 0; c < C; ++c)
            if (dense[r * C + c])
                bit_set(M, ldw, r, c);
}

void or_unpack_bits(const uint64_t *M, i64 ldw, i64 R, i64 C, uint8_t *dense)
{
    for (i64 r = 0; r < R; ++r)
        for (i64 c = 0; c < C; ++c)
            dense[r * C + c] = (uint8_t)bit_get(M, ldw, r, c);
}

/*
 * Boolean product on bit rows (Section 4, matBool operator*): for each column
 * c of A from the last down, and each row r with A_rc = 1, OR row c of B into
 * row r of the result, block by block.  Rows of the result are independent,
 * so blocks of rows run on separate threads.  nwN = words per row of B and C.
 */
void or_bool_mul_w64(const uint64_t *A, i64 lda, const uint64_t *B, i64 ldb,
                     uint64_t *C, i64 ldc, i64 R, i64 K, i64 nwN, int accumulate)
{
    const i64 RB = 64;
#pragma omp parallel for schedule(dynamic, 1)
    for (i64 r0 = 0; r0 < R; r0 += RB) {
        i64 r1 = r0 + RB < R ? r0 + RB : R;
        if (!accumulate)
            for (i64 r = r0; r < r1; ++r)
                memset(C + r * ldc, 0, (size_t)nwN * sizeof(uint64_t));
        for (i64 c = K - 1; c >= 0; --c) {
            const uint64_t *Bc = B + c * ldb;
            for (i64 r = r0; r < r1; ++r) {
                if (!bit_get(A, lda, r, c))
                    continue;
                uint64_t *Cr = C + r * ldc;
                for (i64 w = 0; w < nwN; ++w)
                    Cr[w] |= Bc[w];
            }
        }
    }
}

/* Warshall's algorithm on bit rows, in place (Section 2; Section 4: "similar"). */
void or_bool_warshall_w64(uint64_t *T, i64 ldt, i64 D)
{
    i64 nw = (D + 63) / 64;
    for (i64 k = 0; k < D; ++k) {
        const uint64_t *Tk = T + k * ldt;
#pragma omp parallel for schedule(static)
        for (i64 i = 0; i < D; ++i) {
            if (i == k || !bit_get(T, ldt, i, k))
                continue;
            uint64_t *Ti = T + i * ldt;
            for (i64 w = 0; w < nw; ++w)
                Ti[w] |= Tk[w];
        }
    }
}

/*
 * Row src of the Boolean closure by reachability (Section 2, graph reading):
 * bit j is 1 iff a path src -> j with at least one edge exists.
 */
void or_bool_closure_row_w64(const uint64_t *A, i64 lda, i64 D, i64 src, uint64_t *row)
{
    i64 nw = (D + 63) / 64;
    i64 *queue = (i64 *)malloc((size_t)D * sizeof(i64));
    i64 qh = 0, qt = 0;
    memset(row, 0, (size_t)nw * sizeof(uint64_t));
    for (i64 v = 0; v < D; ++v)
        if (bit_get(A, lda, src, v)) {
            bit_set(row, 0, 0, v);
            queue[qt++] = v;
        }
    while (qh < qt) {
        i64 u = queue[qh++];
        for (i64 v = 0; v < D; ++v)
            if (bit_get(A, lda, u, v) && !bit_get(row, 0, 0, v)) {
                bit_set(row, 0, 0, v);
                queue[qt++] = v;
            }
    }
    free(queue);
}

/* ------------------------------------------------------------------------ */
/* Encoding (Sections 3 and 4)                                              */
/* ------------------------------------------------------------------------ */

/*
 * Anti-distance entry of an edge of integer length w: δ(a) = S·(1 − a) on D,
 * scaled by S, gives entry = S − w; a length >= S is not distinguished from
 * infinity and becomes 0 (Section 3).  In the weight matrices used here 0
 * means "no edge" and maps to the semiring zero 0.
 */
void or_encode_antidist(const uint32_t *W, i64 n, uint32_t S, uint32_t *out)
{
    for (i64 t = 0; t < n; ++t)
        out[t] = (W[t] == 0 || W[t] >= S) ? 0u : S - W[t];
}

/* ------------------------------------------------------------------------ */
/* Distance matrices (Section 4, the dual form; Conclusion, dransclose)      */
/* ------------------------------------------------------------------------ */

/* Saturating distance addition on {0..S}: min(x + y, S). */
static inline uint32_t dist_plus(uint32_t x, uint32_t y, uint32_t S)
{
    uint64_t s = (uint64_t)x + y;
    return s >= S ? S : (uint32_t)s;
}

/*
 * Distance product ("funny" product, Section 3 remark; Section 4 dual with ∧ in
 * place of ∨ and saturating addition in place of ⊗): Z_ij = min over k of
 * min(X_ik + Y_kj, S), combined by min with Z when accumulating.  S plays the
 * role of infinity (the neutral element of min).
 */
void or_dist_mul(const uint32_t *X, const uint32_t *Y, uint32_t *Z, i64 R, i64 K, i64 N, uint32_t S,
                 int accumulate)
{
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < R; ++i)
        for (i64 j = 0; j < N; ++j) {
            uint32_t z = accumulate ? Z[i * N + j] : S;
            for (i64 k = 0; k < K; ++k) {
                uint32_t d = dist_plus(X[i * K + k], Y[k * N + j], S);
                if (d < z) z = d;
            }
            Z[i * N + j] = z;
        }
}

/*
 * Floyd's algorithm on distances, in place, without setting the diagonal to 0:
 * T_ii ends as the shortest cycle through i ("minimum loop lengths on the
 * diagonal", Conclusion).  Lengths saturate at S.
 */
void or_dist_closure(uint32_t *T, i64 D, uint32_t S)
{
    for (i64 k = 0; k < D; ++k) {
        const uint32_t *Tk = T + k * D;
#pragma omp parallel for schedule(static)
        for (i64 i = 0; i < D; ++i) {
            if (i == k) continue;              /* row k is unchanged in step k */
            uint32_t a = T[i * D + k];
            if (a >= S) continue;
            uint32_t *Ti = T + i * D;
            for (i64 j = 0; j < D; ++j) {
                uint32_t d = dist_plus(a, Tk[j], S);
                if (d < Ti[j]) Ti[j] = d;
            }
        }
    }
}

/*
 * Entrywise operations (Conclusion table): op 0: a & b = min(a, b);
 * op 1: a | b = max(a, b); op 2: a ^ b = |a − b|; op 3: ~a = S − a (b unused).
 * For S = 1 these are the Boolean AND, OR, XOR, NOT.
 */
void or_entrywise(int op, const uint32_t *A, const uint32_t *B, uint32_t *out, i64 n, uint32_t S)
{
    for (i64 t = 0; t < n; ++t) {
        uint32_t a = A[t], b = B ? B[t] : 0;
        switch (op) {
        case 0: out[t] = a < b ? a : b; break;
        case 1: out[t] = a > b ? a : b; break;
        case 2: out[t] = a > b ? a - b : b - a; break;
        default: out[t] = S - a; break;
        }
    }
}
