/*
 * CPU oracle for the PFAC multi-pattern scan (test infrastructure only).
 *
 * This file is test infrastructure: only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark use it. The product never links it, and
 * it shares no code, header or table with the CUDA library.
 *
 * What is computed (Sections II-B and II-C of the paper): a set of patterns P
 * and a text T; a walk starts at every byte of T, follows the pattern trie
 * while the text keeps matching and stops at the first mismatch (parallel
 * failure-less Aho-Corasick, one walk per start position). For every start
 * position i the oracle reports
 *   ids[i]  = id of the longest pattern p with T[i .. i+|p|) == p, or -1;
 *   count  += number of patterns that occur at i;
 * where a pattern's id is the index of its first occurrence in the input list
 * (a later duplicate adds nothing). It also counts trie lookups: one per
 * attempted transition, i.e. depth reached + 1 when the walk stopped on a
 * mismatch before the text's end, depth reached when it ran into the end.
 *
 * Two independent implementations:
 *   oracle_naive  the definition itself: every pattern compared at every
 *                 position (the pin for everything else; slow);
 *   oracle_pfac   the PFAC walk over a plain pointer trie whose nodes keep an
 *                 unsorted singly linked list of (byte, child) edges, built by
 *                 inserting one pattern at a time (trie construction, step I
 *                 of Section III; numbering is irrelevant to the outputs).
 *
 * The all-matches form (every occurrence, not only the longest per position;
 * Sections II-B and II-C ask for all matches) lists each (position, pattern
 * id, pattern length) in the order: position ascending, then the longer
 * pattern first. oracle_naive_all and oracle_pfac_all compute it the same two
 * independent ways.
 *
 * Plain C99, no threads; callers split position ranges across threads.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* The definition (Section II-B: find every pattern of P in T).             */
/* ------------------------------------------------------------------------ */

/* Longest-match id, match count and lookup count over start positions
 * [i0, i1) of text[0, len). Pattern j is pat[off[j] .. off[j+1]).
 * Returns 0, or -1 if a pattern is empty (the empty string has no place in
 * a failure-less walk, which must consume a byte before it can match). */
int oracle_naive(const uint8_t *pat, const int64_t *off, int32_t npat,
                 const uint8_t *text, int64_t len, int64_t i0, int64_t i1,
                 int32_t *ids, int64_t *count, int64_t *lookups)
{
    int64_t cnt = 0, look = 0;
    for (int32_t j = 0; j < npat; ++j)
        if (off[j + 1] <= off[j]) return -1;
    for (int64_t i = i0; i < i1; ++i) {
        int32_t best = -1;
        int64_t best_len = 0;
        int64_t deepest = 0; /* longest common prefix of T[i..] with any p */
        for (int32_t j = 0; j < npat; ++j) {
            const uint8_t *p = pat + off[j];
            int64_t L = off[j + 1] - off[j];
            int64_t m = 0;
            while (m < L && i + m < len && text[i + m] == p[m]) ++m;
            if (m > deepest) deepest = m;
            if (m == L) {
                /* p occurs at i; duplicates are counted once (below) */
                int dup = 0;
                for (int32_t q = 0; q < j && !dup; ++q) {
                    int64_t Lq = off[q + 1] - off[q];
                    dup = (Lq == L) && memcmp(pat + off[q], p, (size_t)L) == 0;
                }
                if (dup) continue;
                ++cnt;
                if (L > best_len) { best_len = L; best = j; }
            }
        }
        if (ids) ids[i - i0] = best;
        look += deepest + (i + deepest < len ? 1 : 0);
    }
    if (count) *count = cnt;
    if (lookups) *lookups = look;
    return 0;
}

/* Every occurrence over start positions [i0, i1), by the definition: the
 * distinct patterns occurring at each position, sorted longest first (two
 * patterns occurring at one position are prefixes of each other, so their
 * lengths differ). Writes entries k < cap of pos/id/plen and returns the
 * number of occurrences in *n; -1 for an empty pattern or out of memory. */
int oracle_naive_all(const uint8_t *pat, const int64_t *off, int32_t npat,
                     const uint8_t *text, int64_t len, int64_t i0, int64_t i1,
                     int64_t *pos, int32_t *id, int32_t *plen, int64_t cap, int64_t *n)
{
    int64_t k = 0;
    int32_t *hit = malloc(sizeof(int32_t) * (size_t)(npat > 0 ? npat : 1));
    if (!hit) return -1;
    for (int32_t j = 0; j < npat; ++j)
        if (off[j + 1] <= off[j]) {
            free(hit);
            return -1;
        }
    for (int64_t i = i0; i < i1; ++i) {
        int32_t nh = 0;
        for (int32_t j = 0; j < npat; ++j) {
            const uint8_t *p = pat + off[j];
            int64_t L = off[j + 1] - off[j];
            if (i + L > len || memcmp(text + i, p, (size_t)L) != 0) continue;
            int dup = 0;
            for (int32_t q = 0; q < j && !dup; ++q) {
                int64_t Lq = off[q + 1] - off[q];
                dup = (Lq == L) && memcmp(pat + off[q], p, (size_t)L) == 0;
            }
            if (dup) continue;
            /* insert keeping lengths descending */
            int32_t a = nh++;
            while (a > 0 && off[hit[a - 1] + 1] - off[hit[a - 1]] < L) {
                hit[a] = hit[a - 1];
                --a;
            }
            hit[a] = j;
        }
        for (int32_t a = 0; a < nh; ++a, ++k) {
            if (k >= cap) continue;
            pos[k] = i;
            id[k] = hit[a];
            plen[k] = (int32_t)(off[hit[a] + 1] - off[hit[a]]);
        }
    }
    free(hit);
    *n = k;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Pointer trie and the PFAC walk (Section II-C; Section III step I).       */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t final_id;   /* id of the pattern ending here, or -1 */
    int32_t first_edge; /* head of this node's edge list, or -1 */
} onode;

typedef struct {
    int32_t child;
    int32_t next;       /* next edge of the same parent, or -1 */
    uint8_t byte;
} oedge;

typedef struct otrie {
    onode *nodes;
    oedge *edges;
    int64_t n_nodes, cap_nodes;
    int64_t n_edges, cap_edges;
    int64_t n_dups;
    int64_t max_len;
} otrie;

static int grow(void **p, int64_t *cap, int64_t need, size_t elt)
{
    if (need <= *cap) return 0;
    int64_t c = *cap ? *cap : 1024;
    while (c < need) c *= 2;
    void *q = realloc(*p, (size_t)c * elt);
    if (!q) return -1;
    *p = q;
    *cap = c;
    return 0;
}

static int32_t new_node(otrie *t)
{
    if (grow((void **)&t->nodes, &t->cap_nodes, t->n_nodes + 1, sizeof(onode)))
        return -1;
    t->nodes[t->n_nodes].final_id = -1;
    t->nodes[t->n_nodes].first_edge = -1;
    return (int32_t)t->n_nodes++;
}

otrie *otrie_new(void)
{
    otrie *t = (otrie *)calloc(1, sizeof(otrie));
    if (!t) return NULL;
    if (new_node(t) < 0) { free(t); return NULL; }   /* the root */
    return t;
}

void otrie_free(otrie *t)
{
    if (!t) return;
    free(t->nodes);
    free(t->edges);
    free(t);
}

/* The child of v on byte b, or -1 (linear scan of the edge list). */
static int32_t child_of(const otrie *t, int32_t v, uint8_t b)
{
    for (int32_t e = t->nodes[v].first_edge; e >= 0; e = t->edges[e].next)
        if (t->edges[e].byte == b) return t->edges[e].child;
    return -1;
}

/* Insert pattern p[0..L) with the given id. Returns 0 when inserted, 1 when
 * the same string was inserted before (the earlier id is kept), -1 for an
 * empty pattern or out of memory. */
int otrie_insert(otrie *t, const uint8_t *p, int64_t L, int32_t id)
{
    if (L <= 0) return -1;
    int32_t v = 0;
    for (int64_t d = 0; d < L; ++d) {
        int32_t c = child_of(t, v, p[d]);
        if (c < 0) {
            c = new_node(t);
            if (c < 0) return -1;
            if (grow((void **)&t->edges, &t->cap_edges, t->n_edges + 1, sizeof(oedge)))
                return -1;
            oedge *e = &t->edges[t->n_edges];
            e->child = c;
            e->byte = p[d];
            e->next = t->nodes[v].first_edge;
            t->nodes[v].first_edge = (int32_t)t->n_edges++;
        }
        v = c;
    }
    if (L > t->max_len) t->max_len = L;
    if (t->nodes[v].final_id >= 0) { ++t->n_dups; return 1; }
    t->nodes[v].final_id = id;
    return 0;
}

int64_t otrie_nodes(const otrie *t) { return t->n_nodes; }
int64_t otrie_edges(const otrie *t) { return t->n_edges; }
int64_t otrie_dups(const otrie *t) { return t->n_dups; }
int64_t otrie_max_len(const otrie *t) { return t->max_len; }

/* Out-degree histogram helper: deg[v] for every node (for CSR invariants). */
void otrie_degrees(const otrie *t, int32_t *deg)
{
    for (int64_t v = 0; v < t->n_nodes; ++v) {
        int32_t d = 0;
        for (int32_t e = t->nodes[v].first_edge; e >= 0; e = t->edges[e].next) ++d;
        deg[v] = d;
    }
}

/* The PFAC scan over start positions [i0, i1) of text[0, len): one walk per
 * start position, continuing while the next text byte has a trie edge and
 * stopping at the first mismatch or at the text's end. Every final node the
 * walk passes is a pattern occurring at i: it adds one to the count, and the
 * deepest one gives ids[i]. */
void oracle_pfac(const otrie *t, const uint8_t *text, int64_t len,
                 int64_t i0, int64_t i1, int32_t *ids, int64_t *count,
                 int64_t *lookups)
{
    int64_t cnt = 0, look = 0;
    for (int64_t i = i0; i < i1; ++i) {
        int32_t v = 0, best = -1;
        int64_t j = i;
        for (;;) {
            if (j >= len) break;          /* text ends: no further lookup */
            ++look;                       /* one lookup for T[j] at node v */
            int32_t c = child_of(t, v, text[j]);
            if (c < 0) break;             /* mismatch: the walk terminates */
            v = c;
            ++j;
            if (t->nodes[v].final_id >= 0) {
                ++cnt;
                best = t->nodes[v].final_id;  /* deeper overwrites shallower */
            }
        }
        if (ids) ids[i - i0] = best;
    }
    if (count) *count = cnt;
    if (lookups) *lookups = look;
}

/* Every occurrence over start positions [i0, i1) by the PFAC walk: the final
 * nodes a walk passes are the patterns occurring at its start, shallowest
 * first; they are listed deepest first. Same output contract as
 * oracle_naive_all; returns -1 when out of memory. */
int oracle_pfac_all(const otrie *t, const uint8_t *text, int64_t len, int64_t i0, int64_t i1,
                    int64_t *pos, int32_t *id, int32_t *plen, int64_t cap, int64_t *n)
{
    int64_t k = 0;
    int32_t *fid = malloc(sizeof(int32_t) * (size_t)(t->max_len + 1));
    int32_t *fl = malloc(sizeof(int32_t) * (size_t)(t->max_len + 1));
    if (!fid || !fl) {
        free(fid);
        free(fl);
        return -1;
    }
    for (int64_t i = i0; i < i1; ++i) {
        int32_t v = 0, nf = 0;
        int64_t j = i;
        while (j < len) {
            int32_t c = child_of(t, v, text[j]);
            if (c < 0) break;
            v = c;
            ++j;
            if (t->nodes[v].final_id >= 0) {
                fid[nf] = t->nodes[v].final_id;
                fl[nf] = (int32_t)(j - i);
                ++nf;
            }
        }
        for (int32_t a = nf - 1; a >= 0; --a, ++k) {
            if (k >= cap) continue;
            pos[k] = i;
            id[k] = fid[a];
            plen[k] = fl[a];
        }
    }
    free(fid);
    free(fl);
    *n = k;
    return 0;
}
