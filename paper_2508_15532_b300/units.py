"""Unit scale of section 3.5.1 (eq. unit_scale): the conversion between the
step's normalised code units (G = c = 1, lengths in GM/c^2) and the cgs
units in which the radiation sector's physics (opacities, the radiation
constant, temperatures) is given.

The black-hole mass M fixes the length and time units, and the accretion rate
Mdot the mass (hence density) unit:

    l_unit = G M / c^2,   t_unit = l_unit / c,   M_unit = Mdot t_unit,
    rho_unit = M_unit / l_unit^3,   u_unit = rho_unit c^2.

Reading: the paper prints rho_unit = M_unit / t_unit^3, which is a density
only where lengths and times share a unit (c = 1); in cgs the density unit is
M_unit / l_unit^3 (= M_unit / (c t_unit)^3), which is what this module uses.

The step itself stays in code units.  This module turns cgs inputs into the
rt_config / rt_set_fluid values:

* absorption coefficients (1/length): alpha_code = alpha_cgs l_unit; an
  absorption law alpha^a = C rho^m T^-p (cgs, T in kelvin) becomes the
  per-cell prefactor kappa of the step's alpha^a = kappa rho^m T^-p in code
  units (rho_exp = m, T_exp = p);
* the scattering coefficient alpha^s = kappa_s rho becomes the per-cell
  alpha_s argument (the step multiplies it by rho);
* the code temperature is p / rho in units of c^2 (the step's T = u_g / Y,
  Y = rho / (Gamma - 1)); in kelvin T_K = T_code mu m_p c^2 / k_B;
* the radiation constant in code units makes a_code T_code^4 the code energy
  density of a_cgs T_K^4: a_code = a_cgs (mu m_p c^2 / k_B)^4 / u_unit;
* intensities: I_cgs = I_code u_unit c (energy flux per steradian).
"""
import math

# cgs constants (CODATA 2018; solar mass from the IAU 2015 nominal G M_sun)
G_CGS = 6.67430e-8
C_CGS = 2.99792458e10
K_B = 1.380649e-16
M_P = 1.67262192369e-24
SIGMA_SB = 5.670374419e-5
A_RAD = 4.0 * SIGMA_SB / C_CGS          # radiation constant, erg cm^-3 K^-4
SIGMA_T = 6.6524587321e-25              # Thomson cross-section, cm^2
M_SUN = 1.3271244e26 / G_CGS            # g


class UnitScale:
    """Code <-> cgs scales for a black hole of M_msun solar masses accreting
    Mdot_cgs grams per second; mu is the mean molecular weight of the gas
    temperature T = mu m_p p / (rho k_B)."""

    def __init__(self, M_msun: float, Mdot_cgs: float, mu: float = 1.0):
        if not (M_msun > 0.0 and Mdot_cgs > 0.0 and mu > 0.0):
            raise ValueError("M, Mdot and mu must be positive")
        self.M = M_msun * M_SUN
        self.Mdot = Mdot_cgs
        self.mu = mu
        self.l_unit = G_CGS * self.M / C_CGS ** 2
        self.t_unit = self.l_unit / C_CGS
        self.M_unit = self.Mdot * self.t_unit
        self.rho_unit = self.M_unit / self.l_unit ** 3
        self.u_unit = self.rho_unit * C_CGS ** 2
        self.T_unit = mu * M_P * C_CGS ** 2 / K_B      # kelvin per code temperature

    # ------------------------------------------------------------ conversions
    def temperature_K(self, T_code):
        return T_code * self.T_unit

    def temperature_code(self, T_K):
        return T_K / self.T_unit

    def arad_code(self) -> float:
        """a_rad of the step's emission a T^4 / (4 pi) in code units."""
        return A_RAD * self.T_unit ** 4 / self.u_unit

    def absorption_prefactor(self, C_cgs: float, rho_exp: float, T_exp: float) -> float:
        """kappa (code) of alpha^a = kappa rho^rho_exp T^-T_exp for the cgs law
        alpha^a = C_cgs rho_cgs^rho_exp T_K^-T_exp (alpha in 1/cm)."""
        return C_cgs * self.rho_unit ** rho_exp * self.T_unit ** (-T_exp) * self.l_unit

    def scattering_coefficient(self, kappa_s_cgs: float) -> float:
        """alpha_s argument (code) of alpha^s = alpha_s rho for the cgs opacity
        kappa_s (cm^2/g): alpha^s_cgs = kappa_s rho_cgs."""
        return kappa_s_cgs * self.rho_unit * self.l_unit

    def intensity_cgs(self, I_code):
        return I_code * self.u_unit * C_CGS

    def mdot_eddington(self, efficiency: float = 0.1) -> float:
        """Eddington accretion rate L_Edd / (efficiency c^2), L_Edd = 4 pi G M m_p c / sigma_T."""
        L = 4.0 * math.pi * G_CGS * self.M * M_P * C_CGS / SIGMA_T
        return L / (efficiency * C_CGS ** 2)

    def config_fields(self) -> dict:
        """The rt_config fields that carry the scale (arad); opacity prefactors
        are per cell (absorption_prefactor, scattering_coefficient)."""
        return {"arad": self.arad_code()}
