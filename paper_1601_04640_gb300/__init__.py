"""GB300-native split-step Crank-Nicolson solver for the dipolar
Gross-Pitaevskii equation (arXiv:1601.04640's method), behind a C ABI."""
