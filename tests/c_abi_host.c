/*
 * The C ABI used from plain C99 (no Python, no C++): host-only entry points
 * of libopf_admm on a two-bus, three-phase feeder built here by hand.
 * Prints "c abi ok" and exits 0 when every check holds; otherwise prints the
 * failed check and exits 1.  Built and run by tests/test_c_abi.py.
 *
 * Checks:
 *   - the record sizes this C compiler lays out equal the library's
 *     (opf_record_size, compiled as C++);
 *   - the fine decomposition's sizes (Section III-A, one component per bus,
 *     line, generator and load) from the phase counts G, B, E, L:
 *       globals  2G + B + 4E + 4L   (pg, qg; w; p/q both directions; pd,
 *                                    qd, pb, qb)
 *       locals   4G + B + 10E + 7L  (the copies each component holds)
 *       rows     2B + 3E + 4L       (balance, line rows, wye load rows);
 *   - every operator of Eq. (closed_2) is a symmetric projector (P P = P)
 *     and bbar lies in its complement (P bbar = 0);
 *   - opf_component_operator on hand-solved rows, and on contradictory rows
 *     (OPF_ERR_INCONSISTENT, the row reduction of Section IV-B);
 *   - invalid arguments come back as status codes with a message.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "opf_admm.h"

static int failures = 0;

#define CHECK(cond)                                                   \
    do {                                                              \
        if (!(cond)) {                                                \
            printf("FAILED line %d: %s\n", __LINE__, #cond);          \
            ++failures;                                               \
        }                                                             \
    } while (0)

static void fill3(double* a, double v) { a[0] = a[1] = a[2] = v; }

int main(void) {
    opf_bus bus[2];
    opf_line line;
    opf_gen gen;
    opf_load load;
    opf_problem* p = NULL;
    opf_dims d;
    int s, i, j, k;

    CHECK(opf_abi_version() == OPF_ABI_VERSION);
    CHECK(opf_record_size(0) == sizeof(opf_bus));
    CHECK(opf_record_size(1) == sizeof(opf_line));
    CHECK(opf_record_size(2) == sizeof(opf_gen));
    CHECK(opf_record_size(3) == sizeof(opf_load));
    CHECK(opf_record_size(4) == sizeof(opf_params));
    CHECK(opf_record_size(5) == sizeof(opf_info));
    CHECK(opf_record_size(6) == sizeof(opf_dims));
    CHECK(strcmp(opf_status_string(OPF_ERR_INCONSISTENT), "OPF_ERR_INCONSISTENT") == 0);

    /* bus 0: the substation (w fixed at 1); bus 1: w in [0.81, 1.21] */
    memset(bus, 0, sizeof bus);
    for (i = 0; i < 2; ++i) {
        bus[i].phases = 7;
        fill3(bus[i].w_lo, i == 0 ? 1.0 : 0.81);
        fill3(bus[i].w_hi, i == 0 ? 1.0 : 1.21);
    }
    memset(&line, 0, sizeof line);
    line.from_bus = 0;
    line.to_bus = 1;
    line.phases = 7;
    line.in_service = 1;
    for (i = 0; i < 3; ++i)
        for (j = 0; j < 3; ++j) {
            line.r[3 * i + j] = i == j ? 0.010 : 0.004;
            line.x[3 * i + j] = i == j ? 0.020 : 0.008;
        }
    fill3(line.b_fr, 0.001);
    fill3(line.b_to, 0.001);
    fill3(line.tap, 1.0);
    fill3(line.p_lo, -10.0);
    fill3(line.p_hi, 10.0);
    fill3(line.q_lo, -10.0);
    fill3(line.q_hi, 10.0);
    memset(&gen, 0, sizeof gen);
    gen.bus = 0;
    gen.phases = 7;
    fill3(gen.pg_lo, -10.0);
    fill3(gen.pg_hi, 10.0);
    fill3(gen.qg_lo, -10.0);
    fill3(gen.qg_hi, 10.0);
    fill3(gen.cost, 1.0);
    memset(&load, 0, sizeof load);
    load.bus = 1;
    load.phases = 7;
    load.conn = 0;
    fill3(load.a, 0.10);
    fill3(load.b, 0.03);

    CHECK(opf_problem_create(bus, 2, &line, 1, &gen, 1, &load, 1, &p) == OPF_OK);
    if (!p) {
        printf("create failed: %s\n", opf_last_error());
        return 1;
    }
    CHECK(opf_get_dims(p, &d) == OPF_OK);
    {
        const int G = 3, B = 6, E = 3, L = 3; /* phase counts */
        CHECK(d.n_global == 2 * G + B + 4 * E + 4 * L);
        CHECK(d.n_local == 4 * G + B + 10 * E + 7 * L);
        CHECK(d.n_comp == 5);
        CHECK(d.n_rows == 2 * B + 3 * E + 4 * L);
        CHECK(d.n_rows_reduced > 0 && d.n_rows_reduced <= d.n_rows);
    }

    {
        int total = 0, n = 0;
        for (s = 0; s < d.n_comp; ++s) {
            double *P, *bbar;
            double err_pp = 0.0, err_sym = 0.0, err_pb = 0.0;
            CHECK(opf_get_operator(p, s, NULL, NULL, &n) == OPF_OK);
            CHECK(n >= 1 && n <= d.max_n);
            total += n;
            P = (double*)malloc(sizeof(double) * n * n);
            bbar = (double*)malloc(sizeof(double) * n);
            CHECK(opf_get_operator(p, s, P, bbar, NULL) == OPF_OK);
            for (i = 0; i < n; ++i) {
                double pb = 0.0;
                for (j = 0; j < n; ++j) {
                    double pp = 0.0;
                    for (k = 0; k < n; ++k) pp += P[i * n + k] * P[k * n + j];
                    err_pp = fmax(err_pp, fabs(pp - P[i * n + j]));
                    err_sym = fmax(err_sym, fabs(P[i * n + j] - P[j * n + i]));
                    pb += P[i * n + j] * bbar[j];
                }
                err_pb = fmax(err_pb, fabs(pb));
            }
            CHECK(err_pp <= 1e-10 && err_sym <= 1e-12 && err_pb <= 1e-10);
            free(P);
            free(bbar);
        }
        CHECK(total == d.n_local);
        CHECK(opf_get_operator(p, d.n_comp, NULL, NULL, &n) == OPF_ERR_INVALID_ARG);
    }
    /* no device state yet: solve is out of order, not a crash */
    {
        opf_params prm;
        opf_info info;
        opf_params_default(&prm);
        CHECK(opf_admm_solve(p, &prm, NULL, &info) == OPF_ERR_STATE);
        CHECK(strlen(opf_last_error()) > 0);
    }
    opf_destroy(p);

    /* rows x1 + x2 = 1 and 2 x1 + 2 x2 = 2: one kept row a = (1, 1);
     * P = I - a a^T / 2, bbar = a / 2 */
    {
        const double A[4] = {1.0, 1.0, 2.0, 2.0};
        const double b_ok[2] = {1.0, 2.0}, b_bad[2] = {1.0, 3.0};
        double P[4], bbar[2];
        int32_t m = -1;
        CHECK(opf_component_operator(A, b_ok, 2, 2, P, bbar, &m) == OPF_OK);
        CHECK(m == 1);
        CHECK(fabs(P[0] - 0.5) < 1e-14 && fabs(P[1] + 0.5) < 1e-14 && fabs(P[2] + 0.5) < 1e-14 &&
              fabs(P[3] - 0.5) < 1e-14);
        CHECK(fabs(bbar[0] - 0.5) < 1e-14 && fabs(bbar[1] - 0.5) < 1e-14);
        CHECK(opf_component_operator(A, b_bad, 2, 2, P, bbar, &m) == OPF_ERR_INCONSISTENT);
        CHECK(strlen(opf_last_error()) > 0);
    }

    /* invalid input */
    CHECK(opf_problem_create(bus, 0, &line, 1, &gen, 1, &load, 1, &p) == OPF_ERR_INVALID_ARG);
    bus[1].phases = 0;
    CHECK(opf_problem_create(bus, 2, &line, 1, &gen, 1, &load, 1, &p) == OPF_ERR_INVALID_ARG);
    bus[1].phases = 7;
    line.to_bus = 0;
    CHECK(opf_problem_create(bus, 2, &line, 1, &gen, 1, &load, 1, &p) == OPF_ERR_INVALID_ARG);
    line.to_bus = 1;
    bus[1].w_lo[0] = 2.0; /* lo > hi */
    CHECK(opf_problem_create(bus, 2, &line, 1, &gen, 1, &load, 1, &p) == OPF_ERR_INVALID_ARG);
    CHECK(opf_get_dims(NULL, &d) == OPF_ERR_INVALID_ARG);

    if (failures) {
        printf("%d check(s) failed\n", failures);
        return 1;
    }
    printf("c abi ok\n");
    return 0;
}
