"""Physical constants used by the oracle.

eps0 and mu0 take the rounded values the paper states were used in both its
code and its analytic references (Test 3, "Physical and numerical parameters
of the joint benchmark" table).  The remaining constants are CODATA values;
the paper prints none of them.
"""

EPS0 = 8.8542e-12          # F/m   (Test 3 parameter table)
MU0 = 1.2566e-6            # H/m   (Test 3 parameter table)
QE = 1.602176634e-19       # C
ME = 9.1093837015e-31      # kg
AMU = 1.66053906660e-27    # kg
M_AR = 39.948 * AMU        # kg, argon atom (the Ar+ ion mass is taken equal)
KB = 1.380649e-23          # J/K
TORR = 133.322368          # Pa

E_EXC = 11.55              # eV, Ar excitation threshold of the argon workloads
E_ION = 15.76              # eV, Ar ionisation threshold
