"""B300-native SPOCK hot path: CUDA kernels behind a C-ABI library (libspock)
and a thin Python binding. Importing the package loads nothing; the binding
lives in paper_2505_12078_b300.spock and the seeded generators in
paper_2505_12078_b300.synth."""
