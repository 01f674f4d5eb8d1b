/* A plain C99 caller of the C-ABI: include/spdinv.h must compile as C and
 * libspdinv.so must link and answer without a GPU for everything that needs
 * none (argument checks, planner queries, the batch split).  Prints one
 * "name value" line per check; tests/test_c_abi.py compares them. */
#include <stddef.h>
#include <stdio.h>
#include <stdint.h>

#include "spdinv.h"

int main(void) {
    int64_t cp[4] = {0, 0, 0, 0};
    int64_t counts[12];
    int64_t ntasks = 0;
    double crit = 0.0;
    uint32_t tasks[16];
    int sizes[5] = {5, 9, 9, 3, 7};
    int owner[5] = {0, 0, 0, 0, 0};
    double load[2] = {0.0, 0.0};
    int64_t chk[3] = {0, 0, 0};
    spdinv_opts o = {0};
    int tiles = 0;
    spdinv_status st;

    printf("version %d\n", spdinv_version());
    printf("potri_n %d\n", (int)spdinv_potri(-1, NULL, 1, NULL, 0));
    printf("potri_lda %d\n", (int)spdinv_potri(10, NULL, 5, NULL, 0));
    printf("potri_null %d\n", (int)spdinv_potri(10, NULL, 10, NULL, 0));
    printf("potri_empty %d\n", (int)spdinv_potri(0, NULL, 1, NULL, 0));
    o.tile = 48;
    printf("potri_ex_tile %d\n", (int)spdinv_potri_ex(10, (double*)16, 10, &o, NULL, 0));
    /* each call before the printf that reads its outputs: the order in which
     * a call's arguments are evaluated is unspecified */
    st = spdinv_dag_critical_path(4, 0, cp);
    printf("critical %d %lld %lld %lld\n", (int)st, (long long)cp[0], (long long)cp[1], (long long)cp[2]);
    st = spdinv_dag_task_counts(4, counts);
    printf("counts %d %lld\n", (int)st, (long long)counts[0]);
    st = spdinv_plan_tasks(128, 32, 0, tasks, 16, &ntasks, &crit);
    printf("plan %d %lld\n", (int)st, (long long)ntasks);
    printf("first_task %u\n", tasks[0]);
    st = spdinv_plan_check(16, 0, chk);
    printf("plan_check %d %lld %lld\n", (int)st, (long long)chk[1], (long long)chk[2]);
    st = spdinv_batch_shard(5, sizes, 2, owner, load);
    printf("shard %d %d %d %d %d %d %.0f %.0f\n", (int)st, owner[0], owner[1], owner[2], owner[3], owner[4],
           load[0], load[1]);
    st = spdinv_slice_tile_order(2300, 1, 1, NULL, NULL, &tiles);
    printf("slice_tiles %d %d\n", (int)st, tiles);
    /* the layout of the options struct, for the binding's copy of it */
    printf("opts_size %d\n", (int)sizeof(spdinv_opts));
    printf("opts_offsets %d %d %d %d %d %d %d %d %d %d %d\n", (int)offsetof(spdinv_opts, tile),
           (int)offsetof(spdinv_opts, ctas_per_sm), (int)offsetof(spdinv_opts, precision),
           (int)offsetof(spdinv_opts, refine_steps), (int)offsetof(spdinv_opts, wait_timeout_s),
           (int)offsetof(spdinv_opts, fault_drop_task), (int)offsetof(spdinv_opts, residual),
           (int)offsetof(spdinv_opts, refine_order), (int)offsetof(spdinv_opts, variant),
           (int)offsetof(spdinv_opts, split_segment), (int)offsetof(spdinv_opts, diag_fp64));
    return 0;
}
