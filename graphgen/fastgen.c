/*
 * Fast input construction for the large synthetic graphs (plain C, OpenMP).
 *
 * Input preparation only; nothing here computes any part of the resistance-distance
 * method. The random draws are the same counter-based SplitMix64 streams as
 * graphgen/rng.py (draw i of stream (seed, stream) is mix(key + (i + 1) * GOLDEN)), so
 * the C and numpy generators produce identical graphs.
 *
 *  - gg_rmat_edges: R-MAT endpoints (Chakrabarti, Zhan and Faloutsos, SDM 2004),
 *    one uniform draw per level per edge, quadrant by the cumulative probabilities.
 *  - gg_csr_from_edges: symmetric CSR from an undirected edge list: self-loops
 *    dropped, both directions stored, columns sorted and duplicates removed per row.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t gg_stream_key(uint64_t seed, uint64_t stream)
{
    uint64_t a = mix(seed + GOLDEN);
    return mix(a ^ stream);
}

static inline double uniform_at(uint64_t key, uint64_t i)
{
    return (double)(mix(key + (i + 1) * GOLDEN) >> 11) * (1.0 / 9007199254740992.0);
}

/* m edges for a 2^scale vertex R-MAT; level l uses stream base_stream + 1000*l. */
void gg_rmat_edges(int scale, int64_t m, double a, double b, double c, uint64_t seed, uint64_t base_stream,
                   int64_t *u, int64_t *v)
{
    uint64_t keys[64];
    for (int l = 0; l < scale; ++l) keys[l] = gg_stream_key(seed, base_stream + 1000ULL * (uint64_t)l);
    const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        int64_t x = 0, y = 0;
        for (int l = 0; l < scale; ++l) {
            const double r = uniform_at(keys[l], (uint64_t)e);
            const int64_t row_bit = r >= ab;
            const int64_t col_bit = (r >= a && r < ab) || r >= abc;
            x = (x << 1) | row_bit;
            y = (y << 1) | col_bit;
        }
        u[e] = x;
        v[e] = y;
    }
}

static int cmp_i32(const void *p, const void *q)
{
    const int32_t a = *(const int32_t *)p, b = *(const int32_t *)q;
    return (a > b) - (a < b);
}

/* Symmetric CSR of n vertices from m undirected edges (u[e], v[e]); self-loops dropped,
 * duplicates removed. row_ptr (n+1) is written; col must hold 2*m entries (the final
 * nnz is row_ptr[n]). Returns nnz. */
int64_t gg_csr_from_edges(int64_t n, int64_t m, const int64_t *u, const int64_t *v, int64_t *row_ptr,
                          int32_t *col)
{
    int64_t *cnt = calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e) {
        if (u[e] == v[e]) continue;
        cnt[u[e]]++;
        cnt[v[e]]++;
    }
    int64_t *pos = malloc(sizeof(int64_t) * ((size_t)n + 1));
    pos[0] = 0;
    for (int64_t i = 0; i < n; ++i) pos[i + 1] = pos[i] + cnt[i];
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)n);
    memcpy(fill, pos, sizeof(int64_t) * (size_t)n);
    for (int64_t e = 0; e < m; ++e) {
        if (u[e] == v[e]) continue;
        col[fill[u[e]]++] = (int32_t)v[e];
        col[fill[v[e]]++] = (int32_t)u[e];
    }
    /* sort and deduplicate each row in place, recording the kept length */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        int32_t *r = col + pos[i];
        const int64_t len = pos[i + 1] - pos[i];
        if (len > 1) qsort(r, (size_t)len, sizeof(int32_t), cmp_i32);
        int64_t k = 0;
        for (int64_t j = 0; j < len; ++j)
            if (k == 0 || r[j] != r[k - 1]) r[k++] = r[j];
        cnt[i] = k;
    }
    /* compact rows */
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t dst = row_ptr[i];
        if (dst != pos[i]) memmove(col + dst, col + pos[i], sizeof(int32_t) * (size_t)cnt[i]);
        row_ptr[i + 1] = dst + cnt[i];
    }
    const int64_t nnz = row_ptr[n];
    free(cnt);
    free(pos);
    free(fill);
    return nnz;
}

/* Barabasi-Albert preferential attachment with the same draws as graphgen.families:
 * a clique on m_attach+1 seed vertices; vertex v >= m_attach+1 picks m_attach targets, each
 * the endpoint at position floor(u * L) of the current endpoint list (L its length), where u
 * is draw k of the stream; after its m_attach picks, the targets and then v (m_attach times)
 * are appended to the list. Writes the directed pick list (src, dst) including the clique;
 * returns the number of pairs (duplicates are removed later). */
int64_t gg_ba_edges(int64_t n, int m_attach, uint64_t seed, uint64_t stream, int64_t *src, int64_t *dst)
{
    const uint64_t key = gg_stream_key(seed, stream);
    const int64_t m0 = m_attach + 1;
    const int64_t cap_ends = m0 * (m0 - 1) + 2 * (n - m0) * (int64_t)m_attach + 16;
    int64_t *ends = malloc(sizeof(int64_t) * (size_t)cap_ends);
    int64_t L = 0, np = 0;
    /* clique edges in numpy's triu order, ends = all a's then all b's */
    for (int64_t i = 0; i < m0; ++i)
        for (int64_t j = i + 1; j < m0; ++j) {
            src[np] = i;
            dst[np] = j;
            ++np;
        }
    for (int64_t k = 0; k < np; ++k) ends[L++] = src[k];
    for (int64_t k = 0; k < np; ++k) ends[L++] = dst[k];
    uint64_t draw = 0;
    for (int64_t v = m0; v < n; ++v) {
        const int64_t Lv = L;
        const int64_t first = np;
        for (int q = 0; q < m_attach; ++q) {
            const double u = uniform_at(key, draw++);
            const int64_t tgt = ends[(int64_t)(u * (double)Lv)];
            src[np] = v;
            dst[np] = tgt;
            ++np;
        }
        for (int q = 0; q < m_attach; ++q) ends[L++] = dst[first + q];
        for (int q = 0; q < m_attach; ++q) ends[L++] = v;
    }
    free(ends);
    return np;
}
