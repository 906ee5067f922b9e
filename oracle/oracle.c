/*
 * oracle.c -- plain, slow, obviously correct CPU oracle for the upper hood.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path calls, links or loads
 * this file: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline
 * (and its reference arm) may use it. It shares no code, header, table or
 * constant with the CUDA library.
 *
 * Problem (paper Section 2, "Wagener's algorithm, CUDA version"): given n
 * points presented left to right, return the corners of their upper hood
 * (upper convex hull), left to right. The lower hood and the convex hull (the
 * paper's title problem, of which Section 2 computes the upper half) follow
 * the same rules below. The paper assumes n = 2^s, no three
 * points collinear, x in [0,1] and no rounding error; this oracle drops those
 * assumptions and fixes the readings below instead.
 *
 * Inputs are integer grid coordinates (kx, ky), 0 <= kx, ky < 2^24, standing
 * for the float32 point (kx * 2^-24, ky * 2^-24). Points are sorted
 * lexicographically by (kx, ky). Every orientation value is computed exactly
 * in int64: differences are below 2^24 in magnitude, products below 2^48 and
 * the determinant below 2^49.
 *
 * Readings where the paper is silent:
 *  - order is lexicographic (x, y), so equal x values are allowed;
 *  - a point equal to an earlier point is never a corner (first occurrence
 *    wins);
 *  - collinear points are not corners: a corner must be a strict right turn;
 *  - any n >= 0 is accepted.
 */
#include <stdint.h>
#include <stddef.h>

/* orient(o, a, b) = det(a - o, b - o): > 0 when b is left of the directed
 * line o -> a (the paper's left_of, Section 2, before the g/f functions). */
static int64_t orient_i64(int64_t ox, int64_t oy, int64_t ax, int64_t ay,
                          int64_t bx, int64_t by)
{
    return (ax - ox) * (by - oy) - (ay - oy) * (bx - ox);
}

/* -1, 0, +1 */
int oracle_orient_sign(int32_t ox, int32_t oy, int32_t ax, int32_t ay,
                       int32_t bx, int32_t by)
{
    int64_t d = orient_i64(ox, oy, ax, ay, bx, by);
    return (d > 0) - (d < 0);
}

/* Batch form: signs[i] = sign(orient(p[3i], p[3i+1], p[3i+2])). */
void oracle_orient_signs(const int32_t *kx, const int32_t *ky, int64_t ntri,
                         int8_t *signs)
{
    for (int64_t t = 0; t < ntri; ++t) {
        int64_t o = 3 * t, a = o + 1, b = o + 2;
        signs[t] = (int8_t)oracle_orient_sign(kx[o], ky[o], kx[a], ky[a],
                                              kx[b], ky[b]);
    }
}

/*
 * Upper hood by Andrew's monotone chain (a named published method; the
 * textbook lexicographic upper-hull scan). Scan the points left to right,
 * keeping the corners found so far on a stack:
 *   1. skip the point if it equals the stack top (an exact repeat);
 *   2. while the stack holds >= 2 corners o, a and orient(o, a, b) >= 0
 *      (b is left of or on the line o -> a, so a is not a strict right
 *      turn), pop a;
 *   3. push b.
 * Writes the input indices of the corners to out[0..h) and returns h.
 */
int64_t oracle_upper_hull(const int32_t *kx, const int32_t *ky, int64_t n,
                          int32_t *out)
{
    int64_t h = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (h > 0 && kx[out[h - 1]] == kx[i] && ky[out[h - 1]] == ky[i])
            continue;
        while (h >= 2) {
            int32_t o = out[h - 2], a = out[h - 1];
            if (orient_i64(kx[o], ky[o], kx[a], ky[a], kx[i], ky[i]) >= 0)
                --h;
            else
                break;
        }
        out[h++] = (int32_t)i;
    }
    return h;
}

static int lex_less(const int32_t *kx, const int32_t *ky, int64_t i, int64_t j)
{
    return kx[i] < kx[j] || (kx[i] == kx[j] && ky[i] < ky[j]);
}

/*
 * Brute force, O(n^3), a second and independent definition of the same set:
 * point i is a corner iff it is the first occurrence of its coordinates and
 * there is no pair a, b with p_a <lex p_i <lex p_b and orient(p_a, p_b, p_i)
 * <= 0 (p_i on or below the segment p_a p_b). Meant for n <= a few hundred.
 */
int64_t oracle_upper_hull_brute(const int32_t *kx, const int32_t *ky,
                                int64_t n, int32_t *out)
{
    int64_t h = 0;
    for (int64_t i = 0; i < n; ++i) {
        int corner = 1;
        for (int64_t j = 0; j < i && corner; ++j)
            if (kx[j] == kx[i] && ky[j] == ky[i])
                corner = 0;
        for (int64_t a = 0; a < n && corner; ++a) {
            if (!lex_less(kx, ky, a, i))
                continue;
            for (int64_t b = 0; b < n; ++b) {
                if (!lex_less(kx, ky, i, b))
                    continue;
                if (orient_i64(kx[a], ky[a], kx[b], ky[b], kx[i], ky[i]) <= 0) {
                    corner = 0;
                    break;
                }
            }
        }
        if (corner)
            out[h++] = (int32_t)i;
    }
    return h;
}

/*
 * Batched form: sets s = 0..num_sets-1 occupy [offsets[s], offsets[s+1]).
 * Set s writes its local corner indices at out[offsets[s] ...] and its count
 * at counts[s].
 */
void oracle_upper_hull_batched(const int32_t *kx, const int32_t *ky,
                               const int64_t *offsets, int64_t num_sets,
                               int32_t *out, int32_t *counts)
{
    for (int64_t s = 0; s < num_sets; ++s) {
        int64_t a = offsets[s], n = offsets[s + 1] - a;
        counts[s] = (int32_t)oracle_upper_hull(kx + a, ky + a, n, out + a);
    }
}

/*
 * Lower hood by the same monotone chain (the lower half of Andrew's method):
 * scan left to right; skip a repeat of the stack top; before pushing b, pop
 * the top a (with o below it) while orient(o, a, b) <= 0, i.e. while a is
 * not a strict left turn. The chain runs from the first point to the
 * first occurrence of the last point; a last column of several points gives
 * a vertical last edge. Writes the corner indices to out[0..h), returns h.
 */
int64_t oracle_lower_hull(const int32_t *kx, const int32_t *ky, int64_t n,
                          int32_t *out)
{
    int64_t h = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (h > 0 && kx[out[h - 1]] == kx[i] && ky[out[h - 1]] == ky[i])
            continue;
        while (h >= 2) {
            int32_t o = out[h - 2], a = out[h - 1];
            if (orient_i64(kx[o], ky[o], kx[a], ky[a], kx[i], ky[i]) <= 0)
                --h;
            else
                break;
        }
        out[h++] = (int32_t)i;
    }
    return h;
}

/*
 * Brute force of the lower hood, O(n^3): point i is a corner iff it is the
 * first occurrence of its coordinates and there is no pair a, b with
 * p_a <lex p_i <lex p_b and orient(p_a, p_b, p_i) >= 0 (p_i on or above the
 * segment p_a p_b).
 */
int64_t oracle_lower_hull_brute(const int32_t *kx, const int32_t *ky,
                                int64_t n, int32_t *out)
{
    int64_t h = 0;
    for (int64_t i = 0; i < n; ++i) {
        int corner = 1;
        for (int64_t j = 0; j < i && corner; ++j)
            if (kx[j] == kx[i] && ky[j] == ky[i])
                corner = 0;
        for (int64_t a = 0; a < n && corner; ++a) {
            if (!lex_less(kx, ky, a, i))
                continue;
            for (int64_t b = 0; b < n; ++b) {
                if (!lex_less(kx, ky, i, b))
                    continue;
                if (orient_i64(kx[a], ky[a], kx[b], ky[b], kx[i], ky[i]) >= 0) {
                    corner = 0;
                    break;
                }
            }
        }
        if (corner)
            out[h++] = (int32_t)i;
    }
    return h;
}

/*
 * Convex hull (the paper's title problem, Section 2 computes its upper
 * half): the corners clockwise from the first point, i.e. the upper hood
 * from the first point to the last, then the lower hood from the last point
 * back to the first, without its two ends (they are the upper hood's ends).
 * Corners are strict: collinear points are not corners; repeats count once
 * (first occurrence). `scratch` holds n ints. Returns the corner count.
 */
int64_t oracle_convex_hull(const int32_t *kx, const int32_t *ky, int64_t n,
                           int32_t *out, int32_t *scratch)
{
    int64_t hu = oracle_upper_hull(kx, ky, n, out);
    int64_t hl = oracle_lower_hull(kx, ky, n, scratch);
    int64_t h = hu;
    for (int64_t j = hl - 2; j >= 1; --j)
        out[h++] = scratch[j];
    return h;
}
