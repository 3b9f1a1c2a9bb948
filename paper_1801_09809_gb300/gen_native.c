/*
 * Native helpers for the seeded synthetic input generators (host C, no CUDA).
 *
 * Structure only: R-MAT edge sampling and COO -> CSC conversion with sorted,
 * de-duplicated row indices.  None of the matching arithmetic lives here.
 *
 * Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator: draw k of edge e is mix(seed + (e * 64 + k) * GAMMA).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

#define SM64_GAMMA 0x9E3779B97F4A7C15ULL

/*
 * R-MAT sampling: for each of m edges choose, level by level, one of the four
 * quadrants with probabilities a, b, c, 1-a-b-c (thresholds ta <= tab <= tabc
 * on a 16-bit uniform).  Quadrant b sets the column bit, c the row bit, d both.
 * Samples with row or column >= n are redrawn (scale = ceil(log2 n)).
 */
int gen_rmat_edges(uint64_t seed, int32_t scale, int64_t n, int64_t m,
                   uint32_t ta, uint32_t tab, uint32_t tabc,
                   int64_t *rows, int64_t *cols)
{
    for (int64_t e = 0; e < m; ++e) {
        uint64_t ctr = 0;
        for (int attempt = 0; attempt < 100000; ++attempt) {
            int64_t r = 0, c = 0;
            uint64_t bits = 0;
            int avail = 0;
            for (int l = 0; l < scale; ++l) {
                if (avail == 0) {
                    bits = sm64_mix(seed + ((uint64_t)e * 64u + ctr) * SM64_GAMMA);
                    ++ctr;
                    avail = 4;
                }
                uint32_t u = (uint32_t)(bits & 0xFFFFu);
                bits >>= 16;
                --avail;
                int rb = u >= tab;
                int cb = (u >= ta && u < tab) || (u >= tabc);
                r = (r << 1) | rb;
                c = (c << 1) | cb;
            }
            if (r < n && c < n) {
                rows[e] = r;
                cols[e] = c;
                break;
            }
            if (attempt == 99999)
                return -1;
        }
    }
    return 0;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * COO -> CSC.  rows/cols: m entries in [0, n).  colptr: n+1 (out),
 * rowidx: capacity m (out).  Rows end up strictly increasing in each column
 * (duplicates removed).  Returns nnz, or -1 on a bad index.
 */
int64_t gen_csc_from_coo(int64_t n, int64_t m, const int64_t *rows, const int64_t *cols,
                         int32_t *colptr, int32_t *rowidx)
{
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt)
        return -2;
    for (int64_t e = 0; e < m; ++e) {
        if (cols[e] < 0 || cols[e] >= n || rows[e] < 0 || rows[e] >= n) {
            free(cnt);
            return -1;
        }
        cnt[cols[e] + 1]++;
    }
    for (int64_t j = 0; j < n; ++j)
        cnt[j + 1] += cnt[j];
    int64_t *pos = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!pos) {
        free(cnt);
        return -2;
    }
    memcpy(pos, cnt, ((size_t)n + 1) * sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e)
        rowidx[pos[cols[e]]++] = (int32_t)rows[e];
    free(pos);
    int64_t out = 0;
    colptr[0] = 0;
    for (int64_t j = 0; j < n; ++j) {
        int64_t b = cnt[j], e = cnt[j + 1];
        int32_t *seg = rowidx + b;
        int64_t len = e - b;
        if (len > 32) {
            qsort(seg, (size_t)len, sizeof(int32_t), cmp_i32);
        } else {
            for (int64_t x = 1; x < len; ++x) {
                int32_t v = seg[x];
                int64_t y = x - 1;
                while (y >= 0 && seg[y] > v) {
                    seg[y + 1] = seg[y];
                    --y;
                }
                seg[y + 1] = v;
            }
        }
        for (int64_t x = 0; x < len; ++x) {
            if (x > 0 && seg[x] == seg[x - 1])
                continue;
            rowidx[out++] = seg[x];
        }
        colptr[j + 1] = (int32_t)out;
    }
    free(cnt);
    return out;
}
