/* A plain C99 client of libsfhad: the C ABI of include/sfhad.h used from C,
 * with no C++ and no PyTorch.
 *
 *   sfh_client tables            host-only calls (no device): operator and
 *                                basis tables, argument errors
 *   sfh_client residual d p nodes n_elem u.bin Ja.bin r.bin
 *                                FP64 volume residual of n_elem elements of
 *                                3D/2D Euler (Ranocha's flux): u and Ja read
 *                                from raw double files, r written to one
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "sfhad.h"

static int read_file(const char *path, void *buf, size_t bytes)
{
    FILE *f = fopen(path, "rb");
    if (!f) return 1;
    size_t got = fread(buf, 1, bytes, f);
    fclose(f);
    return got != bytes;
}

static int tables(void)
{
    double xi[9], w[9], D[81], Q1[81], V[81];
    printf("version %d\n", sfh_version());
    if (sfh_operator_tables(4, SFH_NODES_GLL, xi, w, D, Q1) != SFH_OK) return 1;
    printf("gll4 xi %.17g %.17g %.17g w %.17g %.17g\n", xi[0], xi[1], xi[2], w[0], w[1]);
    if (sfh_basis_table(3, SFH_NODES_GAUSS, SFH_BASIS_LEGENDRE, V) != SFH_OK) return 1;
    printf("leg3 V00 %.17g V11 %.17g\n", V[0], V[5]);
    sfh_ctx *ctx = NULL;
    sfh_status st = sfh_create(4, 3, SFH_NODES_GLL, 6, SFH_FLUX_EULER_RANOCHA, &ctx);
    printf("bad_create %d %s\n", (int)st, sfh_last_error()[0] ? "msg" : "nomsg");
    st = sfh_basis_table(3, SFH_NODES_GAUSS, (sfh_basis)7, V);
    printf("bad_basis %d\n", (int)st);
    return 0;
}

static int residual(int d, int p, int nodes, long long n_elem, const char *fu, const char *fj, const char *fr)
{
    const int n = p + 1, nvar = d + 2;
    long long nn = 1;
    for (int k = 0; k < d; ++k) nn *= n;
    const size_t ub = (size_t)(n_elem * nvar * nn) * sizeof(double);
    const size_t jb = (size_t)(n_elem * d * d * nn) * sizeof(double);
    double *hu = malloc(ub), *hj = malloc(jb), *hr = malloc(ub);
    void *du = NULL, *dj = NULL, *dr = NULL;
    sfh_ctx *ctx = NULL;
    int rc = 1;
    if (!hu || !hj || !hr || read_file(fu, hu, ub) || read_file(fj, hj, jb)) goto out;
    if (cudaMalloc(&du, ub) != cudaSuccess || cudaMalloc(&dj, jb) != cudaSuccess ||
        cudaMalloc(&dr, ub) != cudaSuccess) goto out;
    if (cudaMemcpy(du, hu, ub, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dj, hj, jb, cudaMemcpyHostToDevice) != cudaSuccess) goto out;
    if (sfh_create(d, p, (sfh_nodes)nodes, nvar, SFH_FLUX_EULER_RANOCHA, &ctx) != SFH_OK) goto out;
    if (sfh_volume_residual(ctx, n_elem, du, (const double *)dj, dr, SFH_FP64, NULL) != SFH_OK) goto out;
    if (sfh_check(ctx, NULL) != SFH_OK) goto out;
    if (cudaMemcpy(hr, dr, ub, cudaMemcpyDeviceToHost) != cudaSuccess) goto out;
    {
        /* the same residual from host buffers on a metric bound once */
        double *hr2 = malloc(ub);
        int same = 0;
        if (hr2 && sfh_bind_metric(ctx, n_elem, hj) == SFH_OK &&
            sfh_volume_residual_host_bound(ctx, n_elem, hu, hr2, SFH_FP64) == SFH_OK)
            same = memcmp(hr, hr2, ub) == 0;
        free(hr2);
        if (!same) goto out;
    }
    {
        FILE *f = fopen(fr, "wb");
        if (!f) goto out;
        rc = fwrite(hr, 1, ub, f) != ub;
        fclose(f);
    }
out:
    if (rc) fprintf(stderr, "residual failed: %s\n", sfh_last_error());
    if (ctx) sfh_destroy(ctx);
    cudaFree(du);
    cudaFree(dj);
    cudaFree(dr);
    free(hu);
    free(hj);
    free(hr);
    return rc;
}

int main(int argc, char **argv)
{
    if (argc >= 2 && strcmp(argv[1], "tables") == 0) return tables();
    if (argc == 9 && strcmp(argv[1], "residual") == 0)
        return residual(atoi(argv[2]), atoi(argv[3]), atoi(argv[4]), atoll(argv[5]), argv[6], argv[7], argv[8]);
    fprintf(stderr, "usage: sfh_client tables | residual d p nodes n_elem u.bin Ja.bin r.bin\n");
    return 2;
}
