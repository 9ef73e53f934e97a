#include "pplbm.h"
#include <stdio.h>
#include <stddef.h>
int main(){printf("%zu %zu %zu %zu %zu %zu %zu\n",sizeof(lbm_lattice_desc), sizeof(lbm_runtime_opts), sizeof(lbm_kernel_stat),sizeof(lbm_info_t), offsetof(lbm_lattice_desc, mrt_rates), sizeof(lbm_server_opts),sizeof(lbm_server_stats));return 0;}