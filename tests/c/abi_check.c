/* Compiles the public header as C (not C++) and calls the host-only entry
 * points of libdctgb through the C ABI: spec query, tables, PSNR from SSE,
 * rate bits and argument errors.  Exit status 0 on success. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "dctgb.h"

static int fails = 0;
#define CHECK(c)                                                      \
    do {                                                              \
        if (!(c)) {                                                   \
            fprintf(stderr, "check failed: %s (line %d)\n", #c, __LINE__); \
            ++fails;                                                  \
        }                                                             \
    } while (0)

int main(void) {
    dct_spec_info info;
    CHECK(dct_spec_query(&info) == DCT_OK);
    CHECK(info.P == 4 && info.N == 6 && info.R == 11 && info.quant_shift == 32 && info.stats_words == 80);
    CHECK(dct_spec_query(NULL) == DCT_ERR_INVALID_ARG);
    CHECK(strlen(dct_last_error()) > 0);

    uint16_t q[64];
    uint32_t m[64];
    int32_t w[64];
    CHECK(dct_tables(50, NULL, 0, 0, q, m, w) == DCT_OK);
    CHECK(q[0] == 16 && q[1] == 11 && q[63] == 99);     /* T.81 Table K.1 at quality 50 */
    CHECK(m[0] == 2097152u);                            /* rint(2^25 / 16) */
    CHECK(w[0] == 2048);                                /* 2^R */
    CHECK(dct_tables(100, NULL, 0, 1, q, NULL, NULL) == DCT_OK && q[0] == 1 && q[63] == 1);
    CHECK(dct_tables(101, NULL, 0, 0, q, m, w) == DCT_ERR_INVALID_ARG);
    uint16_t bad[64];
    for (int i = 0; i < 64; ++i) bad[i] = 300;
    CHECK(dct_tables(0, bad, 64, 0, q, m, w) == DCT_ERR_INVALID_ARG);

    CHECK(fabs(dct_psnr_from_sse(600, 600, 0.0) - 20.0 * log10(255.0)) < 1e-12);
    CHECK(isinf(dct_psnr_from_sse(0, 10, 0.0)));

    uint64_t st[DCT_ENTROPY_WORDS];
    memset(st, 0, sizeof st);
    st[0] = 4; st[3] = 4;          /* DC categories 0 and 3, four each: 8 bits */
    st[16 + 0x00] = 8;             /* eight EOBs: 0 bits */
    st[272] = 12;                  /* amplitude bits */
    CHECK(fabs(dct_entropy_bits(st) - 20.0) < 1e-12);
    /* prefix codes: DC {4, 4} -> 1 bit each; the lone AC symbol -> 1 bit each */
    CHECK(dct_huffman_bits(st) == 12 + 8 + 8);
    st[0] = 1; st[1] = 1; st[2] = 2; st[3] = 4;   /* DC lengths 3, 3, 2, 1: 14 bits */
    CHECK(dct_huffman_bits(st) == 12 + 14 + 8);
    CHECK(dct_huffman_bits(NULL) == 0);

    dct_plan_t plan = NULL;
    dct_plan_desc desc = {0, 10, DCT_LAYOUT_GRAY8, 0, 0};
    CHECK(dct_plan_create(&plan, &desc, NULL) == DCT_ERR_INVALID_ARG && plan == NULL);
    CHECK(dct_compress(NULL, NULL, 1, 50, NULL, 0, NULL, NULL, NULL) == DCT_ERR_INVALID_ARG);
    CHECK(dct_batch_run_noalloc(NULL, 1, DCT_OP_COMPRESS, NULL, NULL) == DCT_ERR_INVALID_ARG);

    if (fails) return 1;
    printf("c abi ok\n");
    return 0;
}
