/*
 * A plain C client of libkc: counts the canonical k-mers of reads given one
 * per line on standard input and prints "key<TAB>count" for the k-mers seen
 * at least min_count times, ascending.  It shows the C ABI used without any
 * Python: pack the ASCII reads, create a job, add the reads, finalize, size
 * the result, dump it.
 *
 *   kc_count K BLOOM_LOG2 MIN_COUNT < reads.txt
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "kc.h"

static int check(kc_status s, const char* what) {
    if (s == KC_OK) return 0;
    fprintf(stderr, "%s: %s: %s\n", what, kc_status_string(s), kc_last_error());
    return 1;
}

int main(int argc, char** argv) {
    if (argc != 4) {
        fprintf(stderr, "usage: %s K BLOOM_LOG2 MIN_COUNT < reads.txt\n", argv[0]);
        return 2;
    }
    const int k = atoi(argv[1]);
    const uint64_t bloom_bits = 1ull << atoi(argv[2]);
    const uint32_t min_count = (uint32_t)atoi(argv[3]);

    /* read all lines: bases concatenated, one offset per read boundary */
    size_t cap = 1 << 20, n = 0, n_reads = 0, off_cap = 1024;
    char* bases = malloc(cap);
    uint64_t* offsets = malloc(off_cap * sizeof(uint64_t));
    if (!bases || !offsets) return 1;
    offsets[0] = 0;
    int c;
    while ((c = getchar()) != EOF) {
        if (c == '\n') {
            if (n_reads + 2 > off_cap && !(offsets = realloc(offsets, (off_cap *= 2) * sizeof(uint64_t)))) return 1;
            offsets[++n_reads] = n;
            continue;
        }
        if (n == cap && !(bases = realloc(bases, cap *= 2))) return 1;
        bases[n++] = (char)c;
    }
    if (n > offsets[n_reads]) { /* last line without a newline */
        if (n_reads + 2 > off_cap && !(offsets = realloc(offsets, (off_cap *= 2) * sizeof(uint64_t)))) return 1;
        offsets[++n_reads] = n;
    }

    uint64_t* packed = calloc((n + 31) / 32 + 1, sizeof(uint64_t));
    uint64_t* n_mask = calloc((n + 63) / 64 + 1, sizeof(uint64_t));
    if (!packed || !n_mask) return 1;
    if (n && check(kc_pack_ascii(bases, n, packed, n_mask), "kc_pack_ascii")) return 1;

    kc_handle h = NULL;
    if (check(kc_create(k, 1, bloom_bits, 4, min_count, &h), "kc_create")) return 1;
    if (check(kc_add_reads(h, 0, packed, offsets, n_mask, n_reads), "kc_add_reads")) return 1;
    if (check(kc_finalize(h), "kc_finalize")) return 1;
    uint64_t n_out = 0;
    if (check(kc_dump(h, NULL, NULL, 0, &n_out), "kc_dump (size)")) return 1;
    uint64_t* keys = malloc((n_out + 1) * sizeof(uint64_t));
    uint32_t* counts = malloc((n_out + 1) * sizeof(uint32_t));
    if (!keys || !counts) return 1;
    if (check(kc_dump(h, keys, counts, n_out, &n_out), "kc_dump")) return 1;
    for (uint64_t i = 0; i < n_out; ++i) printf("%llu\t%u\n", (unsigned long long)keys[i], counts[i]);
    kc_destroy(h);
    free(keys);
    free(counts);
    free(packed);
    free(n_mask);
    free(bases);
    free(offsets);
    return 0;
}
