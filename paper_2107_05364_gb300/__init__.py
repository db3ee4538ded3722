"""GB300-native tile-based micromagnetics: the dense analytical demagnetization
tensor of Bjork et al. (arXiv 2107.05364) applied inside Landau-Lifshitz
time integration, as hand-written CUDA for sm_103a behind a C ABI."""
