/*
 * A plain C user of the geoheat C-ABI (include/geoheat.h): loads a mesh from
 * host memory, solves one source set and writes the distances.  No Python,
 * no PyTorch: the header and libgeoheat.so only.
 *
 * usage: solve_mesh IN OUT SWEEPS FORM FP64
 *   IN   int64 nv, int64 nf, double V[nv][3], int32 F[nf][3], int32 nsrc,
 *        int32 src[nsrc] (native byte order)
 *   OUT  double d[nv]
 *   FORM 0 face, 1 edge
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "geoheat.h"

static int fail(const char *what, gh_status s) {
    fprintf(stderr, "%s failed (%d): %s\n", what, (int)s, gh_last_error());
    return 1;
}

int main(int argc, char **argv) {
    if (argc != 6) {
        fprintf(stderr, "usage: %s IN OUT SWEEPS FORM FP64\n", argv[0]);
        return 2;
    }
    FILE *in = fopen(argv[1], "rb");
    if (!in) { perror(argv[1]); return 2; }
    int64_t nv = 0, nf = 0;
    int32_t nsrc = 0;
    if (fread(&nv, sizeof nv, 1, in) != 1 || fread(&nf, sizeof nf, 1, in) != 1 || nv <= 0 || nf <= 0) return 2;
    double *V = malloc(sizeof(double) * 3 * (size_t)nv);
    int32_t *F = malloc(sizeof(int32_t) * 3 * (size_t)nf);
    double *d = malloc(sizeof(double) * (size_t)nv);
    if (!V || !F || !d) return 2;
    if (fread(V, sizeof(double), 3 * (size_t)nv, in) != 3 * (size_t)nv) return 2;
    if (fread(F, sizeof(int32_t), 3 * (size_t)nf, in) != 3 * (size_t)nf) return 2;
    if (fread(&nsrc, sizeof nsrc, 1, in) != 1 || nsrc <= 0) return 2;
    int32_t *src = malloc(sizeof(int32_t) * (size_t)nsrc);
    if (!src || fread(src, sizeof(int32_t), (size_t)nsrc, in) != (size_t)nsrc) return 2;
    fclose(in);

    gh_ctx ctx;
    gh_mesh mesh;
    gh_status s = gh_ctx_create(0, 0, &ctx);
    if (s != GH_OK) return fail("gh_ctx_create", s);
    s = gh_mesh_load(ctx, V, nv, F, nf, &mesh);
    if (s != GH_OK) return fail("gh_mesh_load", s);
    gh_params p;
    gh_params_default(&p);
    p.gs_sweeps = atoi(argv[3]);
    p.form = atoi(argv[4]) ? GH_FORM_EDGE : GH_FORM_FACE;
    p.fp64 = atoi(argv[5]);
    s = gh_solve(mesh, src, nsrc, &p, d);
    if (s != GH_OK) return fail("gh_solve", s);

    FILE *out = fopen(argv[2], "wb");
    if (!out || fwrite(d, sizeof(double), (size_t)nv, out) != (size_t)nv) return 2;
    fclose(out);
    gh_mesh_free(mesh);
    gh_ctx_destroy(ctx);
    free(V); free(F); free(d); free(src);
    printf("%s: solved %lld vertices\n", gh_version(), (long long)nv);
    return 0;
}
