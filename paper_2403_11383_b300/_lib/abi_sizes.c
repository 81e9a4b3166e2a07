
#include <stdio.h>
#include "sbs.h"
int main(void) { printf("%zu %zu %zu %zu %zu %zu\n", sizeof(sbs_config), sizeof(sbs_problem),
  sizeof(sbs_result), sizeof(sbs_gait), sizeof(sbs_model), sizeof(sbs_cost)); return 0; }
