/* A plain C client of libhfav.so, built by tests/test_c_abi.py: it uses only
 * include/hfav.h and runs the host-side entry points (no device needed). */
#include <stdio.h>
#include <string.h>

#include "hfav.h"

#define CHECK(x)                                                              \
    do {                                                                      \
        int rc_ = (x);                                                        \
        if (rc_ < 0) {                                                        \
            fprintf(stderr, "%s -> %d: %s\n", #x, rc_, hfav_last_error());   \
            return 1;                                                         \
        }                                                                     \
    } while (0)

int main(void) {
    /* the 2D chain as rule bodies: u -> L (5-point star) -> out */
    enum { U, L, OUT, NF };
    const int rank[NF] = {2, 2, 2};
    const hfav_ref star[5] = {{U, {1, 0, 0}}, {U, {-1, 0, 0}}, {U, {0, 1, 0}}, {U, {0, -1, 0}}, {U, {0, 0, 0}}};
    const hfav_ref grad[4] = {{L, {1, 0, 0}}, {L, {-1, 0, 0}}, {L, {0, 1, 0}}, {L, {0, -1, 0}}};
    const int out_l = L, out_o = OUT;
    const double four = 4.0;
    hfav_rule rules[2];
    memset(rules, 0, sizeof rules);
    rules[0].op = HFAV_OP_EXPR; rules[0].n_in = 5; rules[0].in = star; rules[0].n_out = 1; rules[0].out = &out_l;
    rules[0].n_params = 1; rules[0].params = &four; rules[0].expr = "in0 + in1 + in2 + in3 - p0 * in4";
    rules[1].op = HFAV_OP_EXPR; rules[1].n_in = 4; rules[1].in = grad; rules[1].n_out = 1; rules[1].out = &out_o;
    rules[1].expr = "sqrt((in0 - in1) * (in0 - in1) + (in2 - in3) * (in2 - in3)) * (T)0.5";
    const int axioms[1] = {U}, goals[1] = {OUT}, inout[1] = {0};
    hfav_dag dag;
    memset(&dag, 0, sizeof dag);
    dag.n_fields = NF; dag.field_rank = rank; dag.n_rules = 2; dag.rules = rules;
    dag.n_axioms = 1; dag.axioms = axioms; dag.n_goals = 1; dag.goals = goals;
    dag.ndim = 2; dag.stream_axis = 1; dag.inout = inout;

    hfav_plan_t* a = NULL;
    const int64_t ext[3] = {256, 128, 1};
    CHECK(hfav_analyze(&dag, ext, &a));
    hfav_field_info fi;
    CHECK(hfav_plan_field(a, U, &fi));
    if (fi.halo_lo[0] != 2 || fi.halo_hi[1] != 2) { fprintf(stderr, "halo of u\n"); return 1; }
    hfav_free(a);

    hfav_grid g;
    memset(&g, 0, sizeof g);
    g.extent[0] = 256; g.extent[1] = 128; g.extent[2] = 1;
    g.pitch[0] = 1; g.pitch[1] = 260; g.pitch[2] = 260 * 132;
    g.halo = 2;
    hfav_plan_t* p = NULL;
    CHECK(hfav_plan(&dag, &g, 1, HFAV_F32, HFAV_BC_PERIODIC, "full:smem:32x4", &p));
    static char buf[1 << 20];
    CHECK(hfav_plan_schedule(p, buf, sizeof buf));
    if (strcmp(buf, "full:smem:32x4") != 0) { fprintf(stderr, "schedule %s\n", buf); return 1; }
    CHECK(hfav_plan_source(p, buf, sizeof buf));
    if (!strstr(buf, "hfav_cg_part") || !strstr(buf, "p0 * in4")) { fprintf(stderr, "source\n"); return 1; }
    char tiny[8];
    if (hfav_plan_source(p, tiny, sizeof tiny) != HFAV_EINVAL) { fprintf(stderr, "small buffer\n"); return 1; }
    hfav_free(p);

    /* a rule body that reads a parameter it does not have is refused */
    rules[1].expr = "in0 + p3";
    if (hfav_analyze(&dag, ext, &a) != HFAV_EINVAL) { fprintf(stderr, "bad body accepted\n"); return 1; }
    printf("ok %d\n", hfav_version());
    return 0;
}
