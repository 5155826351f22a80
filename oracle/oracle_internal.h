/* Functions of snn_oracle.c used by snn_oracle_graded.c (oracle only). */
#ifndef ORACLE_INTERNAL_H
#define ORACLE_INTERNAL_H
#include <stdint.h>

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]);
uint64_t oracle_bernoulli_threshold(double p);
int oracle_gscale(double k1, double k2, double k3, double n_conn, double* out);
void oracle_hh_rates(double V, double out[6]);
void oracle_hh_currents(const double p[7], double V, double m, double h, double n, double out[3]);

#endif
