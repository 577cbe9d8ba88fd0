/* Oracle-private helpers.  TEST INFRASTRUCTURE ONLY (see oracle.h). */
#ifndef PCOMP_ORACLE_INTERNAL_H
#define PCOMP_ORACLE_INTERNAL_H
#include <stdint.h>

typedef struct {
  int L[3];
  int per[3];
  int N;
  int32_t *nb;  /* [N][6] neighbour index along +x,-x,+y,-y,+z,-z; -1 if absent */
  uint8_t *vac; /* [N] 1 at a vacancy (missing spin), or NULL */
  int nreal;    /* spins present */
} or_lat;

int or_lat_init(or_lat *L, const int32_t dims[3], const uint8_t periodic[3]);
/* Marks the sites with present[lin] == 0 as vacancies: they lose every bond
 * (their own and their neighbours' towards them).  NULL leaves all present. */
int or_lat_set_present(or_lat *L, const uint8_t *present);
void or_lat_free(or_lat *L);
int or_colour(const or_lat *L, int lin);
int or_coupling(const or_lat *L, const int8_t *J, int lin, int dir);
int64_t or_field(const or_lat *L, const int8_t *J, const int8_t *h, const int8_t *s, int lin);
int64_t or_energy_lat(const or_lat *L, const int8_t *J, const int8_t *h, const int8_t *s);
int64_t or_field_bound(const or_lat *L, const int8_t *J, const int8_t *h);
uint32_t or_half(const uint32_t x[4], int i);
/* (v_i(main) << 16) | v_i(refine) for counter (c0, c1, c2, (ent<<8)|tag). */
uint32_t or_uniform32(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t ent,
                      uint32_t tag_main, uint32_t tag_ref, int i);

#endif
