"""CPU oracle of the best-shift tabu search (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import this
package; the CUDA library never does, and the two share no code.
"""
