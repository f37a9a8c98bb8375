/* Minimal C use of the library: build a grid, set a resting layer with a bump,
 * adapt, take ten CFL steps and print mass and live nodes.  Build against the
 * in-tree library:
 *   gcc -std=c99 -I include examples/step.c -L paper_1404_0405_gb300/_build -lsww -lm -o step */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "sww.h"

static int check(int rc) {
    if (rc != SWW_OK) {
        char msg[256];
        sww_last_error(msg, sizeof msg);
        fprintf(stderr, "sww error %d: %s\n", rc, msg);
        exit(1);
    }
    return rc;
}

int main(void) {
    sww_config cfg = {0};
    cfg.jmin = 3, cfg.jmax = 6, cfg.radius = 6.371e6, cfg.omega = 7.292e-5, cfg.g = 9.80616;
    cfg.H = 1.0e4, cfg.patch = 8, cfg.rk = SWW_RK4, cfg.cfl = 0.8, cfg.eps = 1e-2;
    cfg.precision = SWW_FP64;
    sww_handle* h = NULL;
    check(sww_create(&cfg, NULL, &h));
    int64_t n, e, t, np;
    check(sww_level_sizes(h, cfg.jmax, &n, &e, &t, &np));
    double* xyz = malloc(sizeof(double) * 3 * (size_t)n);
    int32_t* en = malloc(sizeof(int32_t) * 2 * (size_t)e);
    double* dh = malloc(sizeof(double) * (size_t)n);
    double* u = calloc((size_t)e, sizeof(double));
    check(sww_get_grid(h, cfg.jmax, xyz, en));
    for (int64_t i = 0; i < n; ++i) {   /* a 100 m Gaussian bump at (1, 0, 0) */
        const double c = xyz[3 * i] / sqrt(xyz[3 * i] * xyz[3 * i] + xyz[3 * i + 1] * xyz[3 * i + 1] + xyz[3 * i + 2] * xyz[3 * i + 2]);
        const double r = cfg.radius * acos(c > 1 ? 1 : c < -1 ? -1 : c);
        dh[i] = 100.0 * exp(-(r / 5.0e5) * (r / 5.0e5));
    }
    check(sww_set_state(h, dh, u, 0));
    check(sww_adapt(h, -1.0, -1.0));
    check(sww_step(h, -1.0, 10, 1));
    sww_stats st;
    check(sww_stats_get(h, &st));
    int64_t live = 0;
    for (int j = cfg.jmin; j <= cfg.jmax; ++j) live += st.live_nodes[j];
    printf("t = %.0f s, dt = %.1f s, mass = %.15e m^3, live nodes = %lld\n", st.t, st.dt, st.mass, (long long)live);
    sww_destroy(h);
    free(xyz), free(en), free(dh), free(u);
    return 0;
}
