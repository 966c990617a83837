/* A plain C11 user of the library: compiled against include/pyc.h with strict
 * warnings and linked with libpyc.so by tests/test_abi_cpu.py.  It makes only
 * calls that need no GPU (version, spec parsing and run-time compilation,
 * parameter introspection, error reporting) and prints what it saw. */
#include <stdio.h>
#include <string.h>

#include "pyc.h"

int main(void) {
  pyc_map_t m = NULL;
  pyc_reduce_t r = NULL;
  pyc_param_info info;
  pyc_status st;
  int k, np;

  printf("version %s\n", pyc_version());

  st = pyc_map_create("float a, float *x, float b, float *y, float *z", "z[i] = a*x[i] + b*y[i]",
                      "lin_comb_c", NULL, &m);
  if (st != PYC_OK) {
    printf("map_create failed %d: %s\n", (int)st, pyc_last_error());
    return 1;
  }
  np = pyc_map_num_params(m);
  printf("map params %d scalar_bytes %d\n", np, pyc_map_scalar_bytes(m));
  for (k = 0; k < np; ++k) {
    if (pyc_map_param(m, k, &info) != PYC_OK) return 2;
    printf("param %s ptr %d dtype %d off %d slot %d\n", info.name, info.is_pointer, info.dtype,
           info.scalar_offset, info.pointer_slot);
  }
  printf("source has kernel %d\n", strstr(pyc_map_source(m), "pyc_map_lin_comb_c") != NULL);

  st = pyc_reduce_create(PYC_F32, "0", "a+b", "x[i]*y[i]", "float *x, float *y", NULL, &r);
  printf("reduce_create %d out_bytes %d\n", (int)st, st == PYC_OK ? pyc_reduce_out_bytes(r) : -1);

  /* errors come back as statuses with a message */
  {
    pyc_map_t bad = NULL;
    st = pyc_map_create("float *x, float *x", "x[i] = 1", NULL, NULL, &bad);
    printf("bad spec %d null %d msg %d\n", (int)st, bad == NULL, pyc_last_error()[0] != 0);
  }

  if (r) pyc_reduce_destroy(r);
  pyc_map_destroy(m);
  return 0;
}
