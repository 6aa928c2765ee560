/*
 * ffa_oracle_api.h -- declarations of the CPU oracle (test infrastructure only).
 * Used by oracle/ffa_oracle.c and loaded from Python by oracle/__init__.py.
 * Nothing in the CUDA library includes this header.
 */
#ifndef FFA_ORACLE_API_H
#define FFA_ORACLE_API_H
#include <stdint.h>

int oracle_plan(int64_t n, double tsamp, double pmin, double pmax, int bmin, int bmax,
                int max_octaves, double* oct_factor, int64_t* oct_len,
                int max_transforms, int* tr_octave, int* tr_p, int64_t* tr_m,
                int64_t* tr_kept, int64_t* tr_first_trial,
                int* n_octaves, int* n_transforms, int64_t* n_trials);

int64_t oracle_downsampled_length(int64_t n, double f);
int oracle_downsample(const float* x, int64_t n, double f, double* out, int64_t nout);
double oracle_downsampled_variance(double f);

void oracle_ffa_split(int64_t m, int64_t s, int64_t* i, int64_t* j, int64_t* b);
int oracle_ffa_f64(const double* in, int64_t m, int64_t p, double* out);
int oracle_ffa_f32(const float* in, int64_t m, int64_t p, float* out);
double oracle_trial_period(double tau, int64_t p, int64_t m, int64_t s);

int oracle_boxcar_snr(const double* prof, int64_t rows, int64_t p, const int* widths,
                      int nw, double stdnoise, double* snr);
int oracle_boxcar_snr_kind(const double* prof, int64_t rows, int64_t p, const int* widths,
                           int nw, double stdnoise, int kind, double* snr);

int oracle_normalise(const float* x, int64_t n, double* mean, double* stdev, double* out);

int oracle_running_median(const float* x, int64_t n, int64_t w, float* med);
int oracle_running_median_at(const float* x, int64_t n, int64_t w, const int64_t* idx,
                             int64_t nidx, float* med);

int64_t oracle_periodogram(const float* x, int64_t n, double tsamp, double pmin,
                           double pmax, int bmin, int bmax, const int* widths, int nw,
                           const unsigned char* select, double* periods, int* foldbins,
                           double* snr, int64_t cap);
int64_t oracle_periodogram_kind(const float* x, int64_t n, double tsamp, double pmin,
                                double pmax, int bmin, int bmax, const int* widths, int nw,
                                int kind, const unsigned char* select, double* periods,
                                int* foldbins, double* snr, int64_t cap);
#endif
