/* A plain C client of libbtree (include/btree.h), built and run by
 * tests/test_abi.py: the boundary used from C with no Python in between.
 * Without a usable GPU it checks the device-free calls and that bt_create
 * refuses with BT_ECUDA and a message; with one it also prices the
 * single-option N = 20 arithmetic Asian call in FP64 and prints the value. */
#include <stdio.h>
#include <string.h>

#include "btree.h"

int main(void) {
    printf("version %s\n", bt_version());
    if (strcmp(bt_status_str(BT_EBUDGET), "BT_EBUDGET") != 0) return 2;

    bt_option o;
    memset(&o, 0, sizeof(o));
    o.N = 20;
    o.tree_kind = BT_TREE_CRR;
    o.payoff = BT_ASIAN_ARITH_CALL;
    o.S0 = 100.0;
    o.K = 100.0;
    o.rate = 0.05;
    o.sigma = 0.2;
    o.T = 1.0;

    int32_t P = 0, L = 0, ppi = 0;
    int64_t items = 0;
    if (bt_exact_split(&o, BT_PREC_FP64, &P, &L, &ppi, &items) != BT_OK) return 3;
    printf("split P=%d L=%d prefixes_per_item=%d items=%lld\n", P, L, ppi, (long long)items);
    if (P + L != o.N || ppi <= 0 || items < 1) return 4;

    o.N = 41; /* out of range: refused before any device work */
    if (bt_exact_split(&o, BT_PREC_FP64, &P, &L, &ppi, &items) != BT_EINVAL) return 5;
    if (bt_last_error(NULL)[0] == '\0') return 6;
    o.N = 20;

    bt_ctx *ctx = NULL;
    bt_status s = bt_create(0, (size_t)1 << 30, &ctx);
    if (s != BT_OK) {
        printf("no device: %s (%s)\n", bt_status_str(s), bt_last_error(NULL));
        return s == BT_ECUDA && bt_last_error(NULL)[0] != '\0' ? 0 : 7;
    }
    bt_result r;
    s = bt_price_exact(ctx, &o, 1, BT_PREC_FP64, &r, NULL);
    bt_destroy(ctx);
    if (s != BT_OK) return 8;
    printf("value %.15g paths %lld\n", r.value, (long long)r.paths);
    return r.paths == (1ll << 20) && r.value > 0.0 ? 0 : 9;
}
