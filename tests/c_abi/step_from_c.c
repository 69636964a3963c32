/* A plain C consumer of libhgks (no Python): reads a mesh and a state written
 * by the test, evaluates the residual and one implicit step through the C ABI,
 * and writes the results back.
 *
 * Input file (binary, little endian): int64 n_vert, n_cells, n_bface, nvc
 * (vertices per cell: 4 tetrahedra, 8 hexahedra); double xyz[n_vert][3];
 * int64 cells[n_cells][nvc]; int64 bface[n_bface][nvc == 8 ? 4 : 3]; int32
 * btag[n_bface]; hgks_params; double Q[n_cells][5] (caller order).
 * Output file: double R[n_cells][5], then double Q_after_step[n_cells][5]
 * (caller order), then the step's res_l1. */
#include <stdio.h>
#include <stdlib.h>
#include <cuda_runtime.h>
#include "hgks.h"

static int check(hgks_status st, const char *what) {
  if (st != HGKS_OK) {
    fprintf(stderr, "%s: status %d: %s\n", what, (int)st, hgks_last_error());
    return 1;
  }
  return 0;
}

int main(int argc, char **argv) {
  if (argc != 3) { fprintf(stderr, "usage: %s in.bin out.bin\n", argv[0]); return 2; }
  FILE *f = fopen(argv[1], "rb");
  if (!f) return 2;
  int64_t nv, nt, nb, nvc;
  if (fread(&nv, 8, 1, f) != 1 || fread(&nt, 8, 1, f) != 1 || fread(&nb, 8, 1, f) != 1 || fread(&nvc, 8, 1, f) != 1)
    return 2;
  if (nvc != 4 && nvc != 8) return 2;
  const int64_t nfv = nvc == 8 ? 4 : 3;
  double *xyz = malloc(sizeof(double) * 3 * nv);
  int64_t *tet = malloc(sizeof(int64_t) * nvc * nt), *bf = malloc(sizeof(int64_t) * nfv * (nb + 1));
  int32_t *bt = malloc(sizeof(int32_t) * (nb + 1));
  double *Qc = malloc(sizeof(double) * 5 * nt), *Qi = malloc(sizeof(double) * 5 * nt);
  double *out = malloc(sizeof(double) * 5 * nt);
  int64_t *perm = malloc(sizeof(int64_t) * nt);
  hgks_params p;
  if (fread(xyz, 8, 3 * nv, f) != (size_t)(3 * nv) || fread(tet, 8, nvc * nt, f) != (size_t)(nvc * nt) ||
      fread(bf, 8, nfv * nb, f) != (size_t)(nfv * nb) || fread(bt, 4, nb, f) != (size_t)nb ||
      fread(&p, sizeof(p), 1, f) != 1 || fread(Qc, 8, 5 * nt, f) != (size_t)(5 * nt))
    return 2;
  fclose(f);

  hgks_mesh mesh = NULL;
  if (check(nvc == 8 ? hgks_mesh_create_hex(xyz, nv, tet, nt, bf, bt, nb, NULL, 0, 1, 0, &mesh, perm)
                     : hgks_mesh_create(xyz, nv, tet, nt, bf, bt, nb, NULL, 0, 1, 0, &mesh, perm),
            "mesh_create"))
    return 1;
  /* caller order [n][5] -> internal component-major [5][n] */
  for (int64_t i = 0; i < nt; i++)
    for (int c = 0; c < 5; c++) Qi[c * nt + i] = Qc[perm[i] * 5 + c];
  double *Qd = NULL, *Rd = NULL;
  if (cudaMalloc((void **)&Qd, sizeof(double) * 5 * nt) != cudaSuccess ||
      cudaMalloc((void **)&Rd, sizeof(double) * 5 * nt) != cudaSuccess)
    return 1;
  cudaMemcpy(Qd, Qi, sizeof(double) * 5 * nt, cudaMemcpyHostToDevice);

  FILE *o = fopen(argv[2], "wb");
  if (!o) return 2;
  if (check(hgks_residual(mesh, &p, Qd, NULL, Rd, NULL, NULL), "residual") || check(hgks_sync(NULL), "sync")) return 1;
  cudaMemcpy(Qi, Rd, sizeof(double) * 5 * nt, cudaMemcpyDeviceToHost);
  for (int64_t i = 0; i < nt; i++)
    for (int c = 0; c < 5; c++) out[perm[i] * 5 + c] = Qi[c * nt + i];
  fwrite(out, 8, 5 * nt, o);

  hgks_step_info info;
  if (check(hgks_gmres_step(mesh, &p, Qd, NULL, NULL, &info, NULL), "gmres_step")) return 1;
  cudaMemcpy(Qi, Qd, sizeof(double) * 5 * nt, cudaMemcpyDeviceToHost);
  for (int64_t i = 0; i < nt; i++)
    for (int c = 0; c < 5; c++) out[perm[i] * 5 + c] = Qi[c * nt + i];
  fwrite(out, 8, 5 * nt, o);
  fwrite(&info.res_l1, 8, 1, o);
  fclose(o);

  cudaFree(Qd);
  cudaFree(Rd);
  check(hgks_mesh_destroy(mesh), "mesh_destroy");
  free(xyz); free(tet); free(bf); free(bt); free(Qc); free(Qi); free(out); free(perm);
  printf("ok %lld cells res_l1 %.6e\n", (long long)nt, info.res_l1);
  return 0;
}
