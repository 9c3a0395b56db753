/*
 * A plain C client of libpermanova (include/permanova.h), used by
 * tests/test_c_client.py: it builds a small seeded problem on the host, asks
 * the library for s_W through the host-buffer entry point (so it needs no
 * CUDA call of its own), and checks every value against s_W written out as
 * its definition (Sec. 2, Algorithm 1's statistic) in double precision.  It
 * also checks that a bad argument comes back as PERMANOVA_EINVAL with a
 * message and that the context keeps working afterwards.
 *
 * Exit status 0 and the line "c client OK" when every check passes.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "permanova.h"

#define N 300
#define P 40
#define K 4

static uint64_t lcg_state = 0x243F6A8885A308D3ull;
static double unit_draw(void) {   /* a seeded draw in [0, 1) (64-bit LCG, Knuth's constants) */
    lcg_state = lcg_state * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(lcg_state >> 11) * (1.0 / 9007199254740992.0);
}

int main(void) {
    static float mat[N * N];
    static uint8_t labels[P * N];
    float w[K];
    double out[P];
    int counts[K] = {0};

    /* points on a line with a group shift: d_ij = |x_i - x_j| */
    double x[N];
    for (int i = 0; i < N; ++i) x[i] = unit_draw() * 10.0;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) mat[i * N + j] = (float)fabs(x[i] - x[j]);
    for (int p = 0; p < P; ++p)
        for (int i = 0; i < N; ++i) labels[p * N + i] = (uint8_t)(unit_draw() * K);
    for (int i = 0; i < N; ++i) counts[labels[i]]++;
    for (int g = 0; g < K; ++g) w[g] = counts[g] ? 1.0f / (float)counts[g] : 0.0f;

    permanova_ctx *ctx = NULL;
    int rc = permanova_create(0, 0, &ctx);
    if (rc != PERMANOVA_OK) {
        fprintf(stderr, "permanova_create: %d %s\n", rc, permanova_last_error(NULL));
        return 1;
    }
    rc = permanova_sW_host(ctx, mat, N, N, labels, PERMANOVA_LABEL_U8, K, P, w, out, NULL);
    if (rc != PERMANOVA_OK) {
        fprintf(stderr, "permanova_sW_host: %d %s\n", rc, permanova_last_error(ctx));
        return 1;
    }
    int bad = 0;
    for (int p = 0; p < P; ++p) {
        double ref = 0.0;   /* sum over pairs i < j in one group of d_ij^2 * w_g */
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j)
                if (labels[p * N + i] == labels[p * N + j]) {
                    const double d = (double)mat[i * N + j];
                    ref += d * d * (double)w[labels[p * N + i]];
                }
        if (!(fabs(out[p] - ref) <= 1e-5 * fabs(ref))) {
            fprintf(stderr, "row %d: library %.17g, definition %.17g\n", p, out[p], ref);
            bad = 1;
        }
    }
    /* a bad argument: n_groups = 0 */
    rc = permanova_sW_host(ctx, mat, N, N, labels, PERMANOVA_LABEL_U8, 0, P, w, out, NULL);
    if (rc != PERMANOVA_EINVAL || permanova_last_error(ctx) == NULL || permanova_last_error(ctx)[0] == 0) {
        fprintf(stderr, "expected EINVAL with a message, got %d\n", rc);
        bad = 1;
    }
    /* the context still works */
    rc = permanova_sW_host(ctx, mat, N, N, labels, PERMANOVA_LABEL_U8, K, 1, w, out, NULL);
    if (rc != PERMANOVA_OK) {
        fprintf(stderr, "call after an error: %d %s\n", rc, permanova_last_error(ctx));
        bad = 1;
    }
    permanova_destroy(ctx);
    if (bad) return 1;
    printf("c client OK\n");
    return 0;
}
